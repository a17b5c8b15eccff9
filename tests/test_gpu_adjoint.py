"""GPU parity of the B-spline diffusion coefficient and of the kappa adjoint.

* Assembly with kappa a cubic B-spline (control values on the device) matches
  the FP64 oracle within 1e-12 (exact and surrogate).
* iga_kappa_gradient matches the oracle gradient obtained by linearity,
  dL/dc_k = ybar^T A(e_k) x, within 1e-10 of the largest component, for the
  exact matrix and the surrogate.
* On the 48^3, p = 3 workload with 16^3 control values, the gradient agrees
  with central finite differences of the GPU forward L(c) = ybar^T A~(c) x to
  1e-6 relative (L is linear in c, so the difference quotient is exact up to
  rounding), and the torch.autograd wrapper returns the same gradients.
"""
import numpy as np
import pytest

import iga_workloads as W
import oracle
from oracle import adjoint as adj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def iga():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_06971_gb300 as m
    m.load()
    return m


def _bs(dim, p, n_el, nctrl, seed=0, amp=0.04):
    return W.Problem(dim=dim, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="bspline3",
                     kappa_nctrl=nctrl, kappa_ctrl=W.lognormal_ctrl(nctrl, seed=seed))


SMALL = [
    (_bs(2, 2, (9, 8), (5, 6), seed=2), 3, 3),
    (_bs(2, 3, (16, 14), (7, 5), seed=4), 2, 3),
    (_bs(3, 2, (5, 6, 5), (4, 5, 4), seed=5), 2, 3),
    (_bs(3, 3, (8, 7, 9), (4, 4, 5), seed=6), 2, 3),
]
IDS = ["2d_p2", "2d_p3", "3d_p2", "3d_p3"]


def _vec(prob, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(prob.N), rng.standard_normal(prob.N)


@pytest.mark.parametrize("prob,M,q", SMALL, ids=IDS)
def test_bspline_kappa_assembly(iga, prob, M, q):
    A = iga.assemble_exact(prob)
    assert oracle.relative_entry_error(A.values_host(), oracle.exact_matrix(prob)) <= TOL64
    A.destroy()
    B = iga.assemble_surrogate(prob, M, q)
    assert oracle.relative_entry_error(B.values_host(), oracle.surrogate_matrix(prob, M, q)) <= TOL64
    B.destroy()


@pytest.mark.parametrize("kind", ["exact", "common"])
@pytest.mark.parametrize("prob,M,q", SMALL, ids=IDS)
def test_kappa_gradient_matches_oracle(iga, prob, M, q, kind):
    if prob.dim == 3 and prob.p == 3 and kind == "common":
        pytest.skip("oracle by linearity needs one surrogate per control value; covered by the 2-D and p = 2 cases")
    ybar, x = _vec(prob, 11)
    Mk = 0 if kind == "exact" else M
    if kind == "exact":      # the quadrature route (pinned against the linearity route on the CPU)
        ref = adj.exact_kappa_gradient_quadrature(prob, ybar, x)
    else:
        ref = adj.kappa_gradient(prob, kind, M, q, ybar, x)
    got = iga.kappa_gradient(prob, torch.from_numpy(ybar).cuda(), torch.from_numpy(x).cuda(), Mk, q).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_kappa_gradient_empty_omega_is_exact(iga):
    prob = _bs(2, 3, (9, 10), (5, 5), seed=1)          # m = 12: Omega~ empty, surrogate = exact
    ybar, x = _vec(prob, 3)
    y, xx = torch.from_numpy(ybar).cuda(), torch.from_numpy(x).cuda()
    g0 = iga.kappa_gradient(prob, y, xx, 0, 3)
    g1 = iga.kappa_gradient(prob, y, xx, 4, 3)
    assert (g0 - g1).abs().max().item() <= 1e-12 * g0.abs().max().item()


def test_kappa_gradient_rejects_other_kappa(iga):
    prob = W.CFG_2D_P2.problem
    v = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
    with pytest.raises(iga.IgaError) as ei:
        iga.kappa_gradient(prob, v, v, 0, 3)
    assert ei.value.code == -1


def _loss(iga, prob, M, q, ctrl, y, x):
    A = iga.assemble_surrogate(prob, M, q, kappa_ctrl=ctrl) if M else iga.assemble_exact(prob, kappa_ctrl=ctrl)
    val = torch.dot(y, A.apply(x)).item()
    A.destroy()
    return val


@pytest.mark.parametrize("M", [0, 8])
def test_full_size_gradient_matches_finite_differences(iga, M):
    wl = W.CFG_3D_P3_BSPLINE
    prob = wl.problem
    rng = np.random.default_rng(21)
    y = torch.from_numpy(rng.standard_normal(prob.N)).cuda()
    x = torch.from_numpy(rng.standard_normal(prob.N)).cuda()
    ctrl = torch.tensor(prob.kappa_ctrl, dtype=torch.float64, device="cuda")
    g = iga.kappa_gradient(prob, y, x, M, wl.q, kappa_ctrl=ctrl)
    gmax = g.abs().max().item()
    nc = ctrl.numel()
    ks = list(rng.choice(nc, 6, replace=False)) + [int(g.abs().argmax().item())]
    for k in ks:
        h = 1e-3 * ctrl[k].item()
        cp, cm = ctrl.clone(), ctrl.clone()
        cp[k] += h
        cm[k] -= h
        fd = (_loss(iga, prob, M, wl.q, cp, y, x) - _loss(iga, prob, M, wl.q, cm, y, x)) / (2 * h)
        assert abs(fd - g[k].item()) <= 1e-6 * max(abs(g[k].item()), 1e-3 * gmax), (k, fd, g[k].item())
    # Euler's identity: L is linear in c
    L = _loss(iga, prob, M, wl.q, ctrl, y, x)
    assert abs(torch.dot(ctrl, g).item() - L) <= 1e-9 * abs(L) + 1e-12 * (ctrl.abs() * g.abs()).sum().item()


def test_autograd_function(iga):
    prob, M, q = SMALL[0]
    ctrl = torch.tensor(prob.kappa_ctrl, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal(prob.N)).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.standard_normal(prob.N)).cuda()
    y = iga.stiffness_apply(ctrl, x, prob, M, q)
    loss = torch.dot(w, y)
    gc, gx = torch.autograd.grad(loss, (ctrl, x))
    ref_c = adj.kappa_gradient(prob, "common", M, q, w.cpu().numpy(), x.detach().cpu().numpy())
    assert np.abs(gc.cpu().numpy() - ref_c).max() <= 1e-10 * np.abs(ref_c).max()
    S = oracle.surrogate_matrix(prob, M, q)
    ref_x = oracle.apply(S, prob, w.cpu().numpy())              # A~^T w = A~ w
    assert np.abs(gx.cpu().numpy() - ref_x).max() <= 1e-12 * np.abs(S).max() * np.abs(w.cpu().numpy()).max() * prob.S


@pytest.mark.parametrize("M", [8, 0])
def test_autograd_half_norm_loss_directional_fd(iga, M):
    """L = 0.5 y^T y with y = A~(c) x through the autograd wrapper, on the 48^3 p = 3
    workload with 16^3 control values: the gradient agrees with central differences
    (h = 1e-6, FP64) along 32 random directions in (c, x) to 1e-6 relative, plus the
    rounding of the difference quotient itself, 8 eps |L| / (2h) (L is a quartic
    polynomial along the line, so the truncation error is O(h^2) and negligible)."""
    wl = W.CFG_3D_P3_BSPLINE
    prob = wl.problem
    rng = np.random.default_rng(31)
    c0 = torch.tensor(prob.kappa_ctrl, dtype=torch.float64, device="cuda")
    x0 = torch.from_numpy(rng.standard_normal(prob.N)).cuda()
    c = c0.clone().requires_grad_(True)
    x = x0.clone().requires_grad_(True)
    y = iga.stiffness_apply(c, x, prob, M, wl.q)
    L = 0.5 * torch.dot(y, y)
    gc, gx = torch.autograd.grad(L, (c, x))

    def loss(cc, xx):
        with torch.no_grad():
            yy = iga.stiffness_apply(cc, xx, prob, M, wl.q)
            return 0.5 * torch.dot(yy, yy).item()

    h = 1e-6
    fd_round = 8 * np.finfo(np.float64).eps * abs(L.item()) / (2 * h)
    for _ in range(32):
        dc = torch.from_numpy(rng.standard_normal(c0.numel())).cuda()
        dx = torch.from_numpy(rng.standard_normal(prob.N)).cuda()
        fd = (loss(c0 + h * dc, x0 + h * dx) - loss(c0 - h * dc, x0 - h * dx)) / (2 * h)
        an = (torch.dot(gc, dc) + torch.dot(gx, dx)).item()
        assert abs(fd - an) <= 1e-6 * abs(an) + fd_round, (fd, an, fd_round)
