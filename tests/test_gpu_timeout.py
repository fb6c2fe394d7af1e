"""Bounded device waits: every spin-wait of the pipelined kernels gives up
after a limit, records a timeout and returns, so that the CUDA context
stays usable.  feast_selftest_wait_timeout runs that give-up path on a wait
that nothing completes (no fault, no hang: the limit ends it)."""

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def F():
    import paper_0901_2665_gb300 as mod
    return mod


def test_bounded_wait_gives_up_and_the_handle_stays_usable():
    h = F().Handle()
    for polls in (1, 1 << 12):
        with pytest.raises(F().FeastError) as ei:
            h.feast_selftest_wait_timeout(polls)
        assert ei.value.status == F().FEAST_ERR_TIMEOUT
        assert "bounded device wait gave up" in str(ei.value)
    # the same handle and context keep working: a 27-point product afterwards
    # equals the oracle's
    op = workloads.q1_operator(6, 5, 4, workloads.gaussian_potential(2, 3, 6, 5, 4))
    X = np.random.default_rng(5).standard_normal((op.N, 3))
    Y = torch.zeros((3, op.N), dtype=torch.float64, device="cuda")
    h.feast_stencil_apply(6, 5, 4, torch.from_numpy(np.ascontiguousarray(op.A27)).cuda(),
                          torch.from_numpy(np.ascontiguousarray(X.T)).cuda(), Y, 3)
    ref = oracle.assemble(op.A27, 6, 5, 4) @ X
    assert np.abs(Y.cpu().numpy().T - ref).max() <= 1e-13 * np.abs(ref).max()


def test_selftest_argument_errors():
    h = F().Handle()
    for polls in (0, -1, (1 << 26) + 1):
        with pytest.raises(F().FeastError) as ei:
            h.feast_selftest_wait_timeout(polls)
        assert ei.value.status == F().FEAST_ERR_ARG
