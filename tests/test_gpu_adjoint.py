"""GPU parity of the hand-written POD adjoint (pylom_pod_backward behind a
torch.autograd.Function) against the oracle's closed-form gradient of the
truncated-POD reconstruction loss, against central finite differences of
the oracle's forward, and against torch.linalg.svd autograd."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda").t()


def _loss_torch(X, w, U):
    """L = || Y_w - U U^T Y_w ||_F^2 with Y_w = sqrt(w) X (no mean)."""
    Yw = X.double() * torch.sqrt(w)[:, None] if w is not None else X.double()
    return torch.sum((Yw - U @ (U.T @ Yw)) ** 2)


def test_adjoint_matches_closed_form_and_finite_differences():
    # N = 512, M = 16, r = 4, binary64; separated spectrum s_i = 10^(-6 i / 15)
    N, M, r = 512, 16, 4
    X, w, s = synth.known_spectrum(N, M, weights=True, seeds=(7, 8, 9))
    Xd = _dev(X).requires_grad_(True)
    wd = torch.from_numpy(w).cuda()
    U, S, VT = pg.pod_autograd(Xd, r, w=wd, remove_mean=False, leaf_rows=64)
    L = _loss_torch(Xd, wd, U)
    L.backward()
    G = Xd.grad.cpu().numpy()
    L_ref, G_ref = oracle.pod_loss_grad(X, r, w=w, remove_mean=False)
    assert L.item() == pytest.approx(L_ref, rel=1e-9, abs=1e-12 * np.sum(s ** 2))
    rel = np.linalg.norm(G - G_ref) / np.linalg.norm(G_ref)
    assert rel <= 1e-6, rel
    h = 1e-6 * np.abs(X).max()
    rng = np.random.default_rng(10)
    for _ in range(12):
        n, m = int(rng.integers(N)), int(rng.integers(M))
        Xp = X.copy(); Xp[n, m] += h
        Xm = X.copy(); Xm[n, m] -= h
        fd = (oracle.pod_loss_grad(Xp, r, w=w, want_grad=False)[0]
              - oracle.pod_loss_grad(Xm, r, w=w, want_grad=False)[0]) / (2 * h)
        assert G[n, m] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(G_ref).max())


def _signed_svd_reference(Yw, r):
    """torch.linalg.svd with the library's sign rule applied (the largest
    |entry| of each right vector positive, lowest index on ties)."""
    U, S, Vh = torch.linalg.svd(Yw, full_matrices=False)
    with torch.no_grad():
        k = torch.argmax(torch.abs(Vh), dim=1)
        sg = torch.sign(Vh[torch.arange(Vh.shape[0]), k])
    return U[:, :r] * sg[None, :r], S, Vh * sg[:, None]


@pytest.mark.parametrize("remove_mean,mode_kind", [(True, pg.MODES_ORTHONORMAL),
                                                   (False, pg.MODES_PHYSICAL)])
def test_adjoint_general_cotangents_match_torch_svd(remove_mean, mode_kind):
    N, M, r = 300, 12, 5
    rng = np.random.default_rng(11)
    X = np.asfortranarray(rng.standard_normal((N, M)) * np.logspace(0, -2, M)[None, :] + 1.0)
    w = synth.log_uniform_weights(N, seed=12)
    gU = rng.standard_normal((N, r)); gS = rng.standard_normal(M); gVT = rng.standard_normal((M, M))
    if remove_mean:
        # mean removal makes Y_w rank M-1: the last singular pair is an
        # arbitrary null direction, and a loss may not depend on it
        gS[-1] = 0.0
        gVT[-1, :] = 0.0
    # ours
    Xd = _dev(X).requires_grad_(True)
    wd = torch.from_numpy(w).cuda()
    U, S, VT = pg.pod_autograd(Xd, r, w=wd, remove_mean=remove_mean, mode_kind=mode_kind, leaf_rows=40)
    L = (torch.sum(U * torch.from_numpy(gU).cuda()) + torch.sum(S * torch.from_numpy(gS).cuda())
         + torch.sum(VT * torch.from_numpy(gVT).cuda()))
    L.backward()
    G = Xd.grad.cpu().numpy()
    # reference: torch.linalg.svd autograd on the CPU in binary64
    Xc = torch.from_numpy(np.array(X)).requires_grad_(True)
    wc = torch.from_numpy(w)
    Y = Xc - Xc.mean(dim=1, keepdim=True) if remove_mean else Xc
    Yw = Y * torch.sqrt(wc)[:, None]
    Ur, Sr, Vhr = _signed_svd_reference(Yw, r)
    if mode_kind == pg.MODES_PHYSICAL:
        Ur = Ur / torch.sqrt(wc)[:, None]
    Lr = (torch.sum(Ur * torch.from_numpy(gU)) + torch.sum(Sr * torch.from_numpy(gS))
          + torch.sum(Vhr * torch.from_numpy(gVT)))
    Lr.backward()
    G_ref = Xc.grad.numpy()
    assert np.allclose(U.detach().cpu().numpy(), Ur.detach().numpy(), atol=1e-10)
    rel = np.linalg.norm(G - G_ref) / np.linalg.norm(G_ref)
    assert rel <= 1e-8, rel


def test_adjoint_full_size_fp32():
    # 4,194,304 x 256 float32 snapshots (six-decade spectrum, weights), r = 20
    N, M, r = 1 << 22, 256, 20
    XT, w, s = synth.known_spectrum_torch(N, M, device="cuda", dtype=torch.float32)
    X = XT.t().detach().requires_grad_(True)
    U, S, VT = pg.pod_autograd(X, r, w=w, remove_mean=False)
    L = _loss_torch(X, w, U)
    L.backward()
    G = X.grad
    assert G.dtype == torch.float32
    with torch.no_grad():
        Yw = X.double() * torch.sqrt(w)[:, None]
        Gc = 2.0 * torch.sqrt(w)[:, None] * (Yw - U @ (U.T @ Yw))
        rel = (torch.linalg.norm(G.double() - Gc) / torch.linalg.norm(Gc)).item()
        # the loss is the spectrum's tail energy
        tail = float(np.sum(S.cpu().numpy()[r:] ** 2))
    assert rel <= 1e-4, rel
    assert L.item() == pytest.approx(tail, rel=1e-6)


def test_adjoint_full_size_matches_torch_svd_autograd():
    # the same 4,194,304 x 256 loss differentiated by torch autograd through
    # torch.linalg.qr and torch.linalg.svd of the 256 x 256 factor, in
    # binary64 (library reference; cuSOLVER's SVD of the whole 4M x 256
    # matrix is refused for its size)
    N, M, r = 1 << 22, 256, 20
    XT, w, s = synth.known_spectrum_torch(N, M, device="cuda", dtype=torch.float32)
    X = XT.t().detach().requires_grad_(True)
    U, S, VT = pg.pod_autograd(X, r, w=w, remove_mean=False)
    _loss_torch(X, w, U).backward()
    G = X.grad.double()
    Xr = XT.t().double().detach().requires_grad_(True)
    Yw = Xr * torch.sqrt(w)[:, None]
    Qr, Rr = torch.linalg.qr(Yw)
    Ur_R, Sr, Vhr = torch.linalg.svd(Rr)
    Ur = Qr @ Ur_R[:, :r]
    Lr = torch.sum((Yw - Ur @ (Ur.T @ Yw)) ** 2)
    Lr.backward()
    with torch.no_grad():
        rel = (torch.linalg.norm(G - Xr.grad) / torch.linalg.norm(Xr.grad)).item()
    assert rel <= 1e-4, rel


# ---------------------------------------------------------------------------
# mixed-precision forward (FP32 modes) and its tcgen05 adjoint
# ---------------------------------------------------------------------------
# FP32 storage and 3xTF32 products leave about 1e-7 relative error in the
# modes; the gradient 2 sqrt(w) (I - U_r U_r^T) Y_w amplifies it by the
# inverse gap (s_r - s_{r+1}) / s_max ~ 0.1 here, and by s_max over the tail
# norm, so 1e-4 (relative Frobenius) leaves a wide margin.
MIXED_GRAD = 1e-4


def test_adjoint_mixed_matches_closed_form():
    N, M, r = 512, 16, 4
    X, w, s = synth.known_spectrum(N, M, weights=True, seeds=(7, 8, 9))
    Xd = _dev(X).float().requires_grad_(True)
    wd = torch.from_numpy(w).cuda()
    U, S, VT = pg.pod_autograd(Xd, r, w=wd, remove_mean=False, leaf_rows=64, prec=pg.PREC_MIXED_3XTF32)
    assert U.dtype == torch.float32
    L = _loss_torch(Xd, wd, U.double())
    L.backward()
    G = Xd.grad.double().cpu().numpy()
    _, G_ref = oracle.pod_loss_grad(Xd.detach().double().cpu().numpy(), r, w=w, remove_mean=False)
    rel = np.linalg.norm(G - G_ref) / np.linalg.norm(G_ref)
    assert rel <= MIXED_GRAD, rel


@pytest.mark.parametrize("remove_mean", [False, True])
def test_adjoint_mixed_matches_fp64_adjoint(remove_mean):
    # general cotangents (dU, dS, dVT) through both adjoints on the same X
    # distinct singular values, so the modes are unique up to sign on both
    # paths, and one decade only: cotangents of every right vector couple all
    # pairs through 1 / (s_j^2 - s_i^2), so the comparison needs every
    # direction resolved at FP32 accuracy (a six-decade spectrum leaves the
    # smallest ones a few percent accurate in FP32)
    N, M, r = 20000, 48, 6
    X = synth.known_spectrum(N, M, s=synth.spectrum(M, decades=1.0), weights=False,
                             seeds=(21, 22, 23))[0].astype(np.float32)
    Xd = _dev(X)
    g = torch.Generator(device="cuda").manual_seed(11)
    dU = torch.randn(N, r, dtype=torch.float64, device="cuda", generator=g)
    dS = torch.randn(M, dtype=torch.float64, device="cuda", generator=g)
    dVT = torch.randn(M, M, dtype=torch.float64, device="cuda", generator=g)
    out = {}
    for prec in (pg.PREC_FP64, pg.PREC_MIXED_3XTF32):
        res = pg.pod(Xd, remove_mean=remove_mean, r_max=r, leaf_rows=2000, prec=prec)
        out[prec] = pg.pod_backward(res, (N, M), None, remove_mean, pg.MODES_ORTHONORMAL, 2000, r,
                                    dU=dU, dS=dS, dVT=dVT).double()
        out[prec, "U"] = res.U.double()
    # both forwards use the same sign rule, so the modes agree column by column
    assert torch.allclose(out[pg.PREC_FP64, "U"], out[pg.PREC_MIXED_3XTF32, "U"], atol=1e-4)
    a, b = out[pg.PREC_FP64], out[pg.PREC_MIXED_3XTF32]
    rel = (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item()
    assert rel <= MIXED_GRAD, rel


def test_adjoint_mixed_full_size_fp32():
    # 4,194,304 x 256 float32 snapshots (six-decade spectrum, weights), r = 20
    N, M, r = 1 << 22, 256, 20
    XT, w, s = synth.known_spectrum_torch(N, M, device="cuda", dtype=torch.float32)
    X = XT.t().detach().requires_grad_(True)
    U, S, VT = pg.pod_autograd(X, r, w=w, remove_mean=False, prec=pg.PREC_MIXED_3XTF32)
    L = _loss_torch(X, w, U.double())
    L.backward()
    G = X.grad
    assert G.dtype == torch.float32
    with torch.no_grad():
        Ud = U.double()
        Yw = X.double() * torch.sqrt(w)[:, None]
        Gc = 2.0 * torch.sqrt(w)[:, None] * (Yw - Ud @ (Ud.T @ Yw))
        rel = (torch.linalg.norm(G.double() - Gc) / torch.linalg.norm(Gc)).item()
        tail = float(np.sum(S.cpu().numpy()[r:] ** 2))
    assert rel <= MIXED_GRAD, rel
    assert L.item() == pytest.approx(tail, rel=1e-5)
