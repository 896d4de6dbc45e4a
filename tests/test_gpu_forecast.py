"""Forward mode (swcl_jvp) and the Gaussian Fisher matrix (swcl_gaussian_fisher) on the GPU
against the oracle (oracle/forecast.py, Sec. 4.3), through the C ABI.

Gates: dC entries as in reading R9 with the floor scaled to the tangent,
    |dC - dC_o| <= tol max(|dC_o|, 1e-3 sqrt(C_ii C_jj) max|dC_o| / max|C_o|),
tol = 1e-10 (FP64) and 1e-4 (bf16x9); Fisher entries relative to the largest, 1e-9 and 1e-3
(the Fisher matrix is a sum of products of two dC, each within its gate)."""
import copy

import numpy as np
import pytest

from gpu_helpers import lib_context, make_ragged_case
from oracle import fftlog as O
from oracle import forecast as F

pytestmark = pytest.mark.gpu

F_SKY = 0.4363


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _one_walker_case():
    w, (tc, tn) = make_ragged_case(n_walk=1, seed=31)
    w = copy.copy(w)
    w.W, w.P, w.amp, w.ell_lists = w.W[0], w.P[0], w.amp[0], None
    return w, (tc, tn)


def _tangents(w, n_dir=4, seed=6):
    """Direction 0: P only; 1: amplitudes only; 2: windows of tracers 1 and 5; 3: all together."""
    rng = np.random.default_rng(seed)
    Pd = np.zeros((n_dir, len(w.k)))
    Ad = np.zeros((n_dir, w.n_tr))
    Wd = np.zeros((n_dir, w.n_tr, w.N))
    Pd[0] = rng.standard_normal(len(w.k)) * w.P
    Ad[1] = rng.standard_normal(w.n_tr)
    Wd[2, [1, 5]] = rng.standard_normal((2, w.N)) * w.W[[1, 5]]
    Pd[3] = rng.standard_normal(len(w.k)) * w.P
    Ad[3] = rng.standard_normal(w.n_tr)
    Wd[3] = rng.standard_normal((w.n_tr, w.N)) * w.W
    return Pd, Ad, Wd


def _modes(ells):
    e = np.asarray(ells, dtype=np.float64)
    edges = np.concatenate([[e[0] - 0.5], 0.5 * (e[1:] + e[:-1]), [e[-1] + 0.5]])
    return (2.0 * e + 1.0) * F_SKY * np.diff(edges)


def _ref():
    w, tapers = _one_walker_case()
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias)
    f = O.forward(g, w.W, w.D, w.P, w.amp, w.B, *tapers)
    Pd, Ad, Wd = _tangents(w)
    J = np.array([F.jvp(g, f, w.D, w.P, w.amp, w.B, *tapers, P_dot=Pd[t], amp_dot=Ad[t], W_dot=Wd[t])
                  for t in range(len(Pd))])
    noise = 1e-3 * np.abs(np.einsum("lii->i", f["C"])) / len(w.ells)
    modes = _modes(w.ells)
    Fo = F.gaussian_quad(f["C"], J, noise, modes)
    return w, tapers, f, (Pd, Ad, Wd), J, noise, modes, Fo


@pytest.fixture(scope="module")
def ref():
    return _ref()


def _jvp_excess(J, Jo, C, tol):
    dg = np.abs(np.einsum("lii->li", C))
    base = np.sqrt(dg[:, :, None] * dg[:, None, :])
    worst = 0.0
    for t in range(len(Jo)):
        floor = 1e-3 * base * np.abs(Jo[t]).max() / np.abs(C).max()
        worst = max(worst, float(np.max(np.abs(J[t] - Jo[t]) / (tol * np.maximum(np.abs(Jo[t]), floor)))))
    return worst


@pytest.mark.parametrize("prec,tol,ftol", [("fp64", 1e-10, 1e-9), ("bf16x9", 1e-4, 1e-3)])
def test_jvp_and_fisher_against_oracle(prec, tol, ftol, ref):
    import paper_2505_22718_gb300 as S
    w, tapers, f, (Pd, Ad, Wd), Jo, noise, modes, Fo = ref
    ctx = lib_context(w, tapers)
    p = S.PRECISIONS[prec]
    C = ctx.compute_cl(p)
    J = ctx.jvp(Pd, Ad, Wd, p)
    assert J.shape == Jo.shape and np.all(np.isfinite(J))
    assert np.array_equal(J, np.transpose(J, (0, 1, 3, 2)))
    ex = _jvp_excess(J, Jo, f["C"], tol)
    Fg = ctx.gaussian_fisher(J, modes, noise)
    fe = float(np.max(np.abs(Fg - Fo)) / np.abs(Fo).max())
    print("%s: jvp excess %.3g  fisher rel %.2e" % (prec, ex, fe))
    assert ex <= 1.0
    assert np.array_equal(Fg, Fg.T)
    assert fe < ftol
    # C left by the forward pass and by the JVP (its base walker) give the same Fisher matrix
    ctx2 = lib_context(w, tapers)
    ctx2.jvp(Pd[:1], None, None, p)
    F2 = ctx2.gaussian_fisher(J, modes, noise)
    assert np.max(np.abs(F2 - Fg)) <= (1e-12 if prec == "fp64" else ftol) * np.abs(Fg).max()
    del C


def test_jvp_is_the_transpose_of_the_vjp_on_device(ref):
    """<C_bar, J v> from swcl_jvp equals <J^T C_bar, v> from swcl_vjp (both on the GPU, FP64)."""
    import paper_2505_22718_gb300 as S
    w, tapers, f, (Pd, Ad, Wd), *_ = ref
    ctx = lib_context(w, tapers)
    rng = np.random.default_rng(17)
    Cb = rng.standard_normal(f["C"].shape)
    ctx.compute_cl(S.SWCL_FP64)
    Pb, Ab, Wb = ctx.vjp(Cb, S.SWCL_FP64)
    J = ctx.jvp(Pd, Ad, Wd, S.SWCL_FP64)
    for t in range(len(Pd)):
        lhs = float(np.sum(Cb * J[t]))
        rhs = float(np.sum(Pb[0] * Pd[t]) + np.sum(Ab[0] * Ad[t]) + np.sum(Wb[0] * Wd[t]))
        assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs)), t


def test_fisher_device_arrays_and_chi2(ref):
    """Device tensors in and out; chi^2 of a perturbation is the one-entry Fisher form."""
    torch = pytest.importorskip("torch")
    import paper_2505_22718_gb300 as S
    w, tapers, f, (Pd, Ad, Wd), Jo, noise, modes, Fo = ref
    ctx = lib_context(w, tapers)
    ctx.compute_cl(S.SWCL_FP64)
    Jd = torch.empty((len(Pd), len(w.ells), w.n_tr, w.n_tr), dtype=torch.float64, device="cuda:0")
    S.swcl_jvp(ctx.ptr, S.SWCL_FP64, len(Pd), Jd, torch.from_numpy(Pd).cuda(),
               torch.from_numpy(Ad).cuda(), torch.from_numpy(Wd).cuda())
    Fd = torch.empty((len(Pd), len(Pd)), dtype=torch.float64, device="cuda:0")
    S.swcl_gaussian_fisher(ctx.ptr, Jd, torch.from_numpy(modes).cuda(), Fd, torch.from_numpy(noise).cuda())
    Fh = ctx.gaussian_fisher(Jd.cpu().numpy(), modes, noise)
    assert np.array_equal(Fd.cpu().numpy(), Fh)
    chi2 = ctx.gaussian_fisher(Jo[2:3], modes, noise)[0, 0]
    want = F.gaussian_quad(f["C"], Jo[2:3], noise, modes)[0, 0]
    assert abs(chi2 - want) <= 1e-9 * want


def test_forecast_argument_and_state_errors(ref):
    import paper_2505_22718_gb300 as S
    w, tapers, f, (Pd, Ad, Wd), Jo, noise, modes, Fo = ref
    ctx = lib_context(w, tapers)
    with pytest.raises(S.SwiftClError):            # no forward pass yet
        ctx.gaussian_fisher(Jo, modes, noise)
    ctx.compute_cl(S.SWCL_FP64)
    with pytest.raises(S.SwiftClError):            # negative noise
        ctx.gaussian_fisher(Jo, modes, -noise)
    ctx.jvp(Pd, None, None, S.SWCL_FP64)
    with pytest.raises(S.SwiftClError):            # the JVP replaced the forward state
        ctx.vjp(np.ones_like(f["C"]), S.SWCL_FP64)
    # two walkers: the JVP is taken at one parameter point
    w2 = copy.copy(w)
    w2.W = np.stack([w.W, w.W])
    w2.P = np.stack([w.P, w.P])
    w2.amp = np.stack([w.amp, w.amp])
    ctx2 = lib_context(w2, tapers)
    with pytest.raises(S.SwiftClError):
        ctx2.jvp(Pd, None, None, S.SWCL_FP64)


@pytest.mark.parametrize("prec", ["fp64", "bf16x9"])
def test_jvp_under_a_memory_budget(prec, wl):
    """The JVP's Delta (base walker and one walker per tangent) in multipole chunks under a
    memory budget gives the same C_dot as without a budget."""
    import paper_2505_22718_gb300 as S
    w0 = wl("n5k_vjp")
    w = copy.copy(w0)
    rng = np.random.default_rng(4)
    Pd = rng.standard_normal((2, len(w.k))) * w.P
    Wd = rng.standard_normal((2, w.n_tr, w.N)) * w.W
    p = S.PRECISIONS[prec]
    ctx = lib_context(w)
    J1 = ctx.jvp(Pd, None, Wd, p)
    held = ctx.query(S.SWCL_Q_WORKSPACE_BYTES)
    es = 8 if prec == "fp64" else 4
    ctx2 = lib_context(w, budget=held - w.n_tr * len(w.ells) * len(w.k) * es // 2)
    J2 = ctx2.jvp(Pd, None, Wd, p)
    assert ctx2.query(S.SWCL_Q_RECOMPUTE) == 1
    assert np.array_equal(J1, J2)
