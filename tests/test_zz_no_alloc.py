"""The allocation-free reduced eigensolve (feast_reduced_eig_noalloc) gives
the same result as the handle-based feast_reduced_eig.

It exists for callers that cannot call cudaMalloc (their device memory is
owned by their own pool or capped at start-up, or an allocation in the middle
of their work is not acceptable), so it keeps its work space in a fixed device
array inside the library.  The test calls it twice in a row through the C-ABI
(the array keeps the previous call's contents, so the second call checks that
nothing stale leaks through), checks an invalid size is refused without any
GPU work, and that a failing call does not poison the next one.  This file is
collected last so a failure here cannot hide the other tests.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem(m, seed, bcond=1e3):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((m, m)))[0]
    BQ = U @ np.diag(np.logspace(0, -np.log10(bcond), m)) @ U.T
    S = rng.standard_normal((m, m))
    return S + S.T, BQ


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def test_noalloc_matches_handle_entry_point_twice():
    import paper_0901_2665_gb300 as F
    h = F.Handle()
    # 128 and 48 run on a thread-block cluster, 16 and 1 on the one-CTA kernel
    for call, (m, seed) in enumerate([(128, 11), (48, 12), (16, 14), (1, 15)]):
        AQ, BQ = _problem(m, seed)
        eps_ref = torch.zeros(m, dtype=torch.float64, device="cuda")
        Phi_ref = torch.zeros((m, m), dtype=torch.float64, device="cuda")
        h.feast_reduced_eig(_dev(AQ), _dev(BQ), m, eps_ref, Phi_ref)
        eps = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
        Phi = torch.full((m, m), np.nan, dtype=torch.float64, device="cuda")
        st = F.feast_reduced_eig_noalloc(_dev(AQ), _dev(BQ), m, eps, Phi)
        assert st == F.FEAST_OK, (call, st)
        e_ref, e = eps_ref.cpu().numpy(), eps.cpu().numpy()
        assert np.abs(e - e_ref).max() <= 1e-10 * np.abs(e_ref).max(), call
        P_ref, P = Phi_ref.cpu().numpy(), Phi.cpu().numpy()
        assert np.abs(P - P_ref).max() <= 1e-10 * np.abs(P_ref).max(), call


def test_noalloc_rejects_oversize_and_recovers_after_failure():
    import paper_0901_2665_gb300 as F
    m = 129
    big = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    out = torch.zeros(m, dtype=torch.float64, device="cuda")
    assert F.feast_reduced_eig_noalloc(big, big, m, out, big) == F.FEAST_ERR_ARG
    # a B_Q of rank m/2 is refused ...
    m = 32
    rng = np.random.default_rng(9)
    V = rng.standard_normal((m, m // 2))
    eps = torch.zeros(m, dtype=torch.float64, device="cuda")
    Phi = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    st = F.feast_reduced_eig_noalloc(_dev(np.eye(m)), _dev(V @ V.T), m, eps, Phi)
    assert st == F.FEAST_ERR_BQ_NOT_SPD
    # ... and the next call starts from a clean status word
    AQ, BQ = _problem(m, 13)
    st = F.feast_reduced_eig_noalloc(_dev(AQ), _dev(BQ), m, eps, Phi)
    assert st == F.FEAST_OK
    import scipy.linalg as sla
    ref = sla.eigh(AQ, BQ)[0]
    assert np.abs(eps.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
