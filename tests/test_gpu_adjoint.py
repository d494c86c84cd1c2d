"""Adjoint gradient of the smoothed line flux (rt_flux_gradient, behind
torch.autograd.Function) against central finite differences of the GPU
forward pipeline and of the FP64 oracle (the CPU reference gradient).

Finite differences use a relative step of 1e-6 (absolute 1e-6 rad for the
angles) at rtol 1e-12, so that the step-size controller's discrete decisions
move F by much less than the difference quotient resolves.  The adjoint is
the exact gradient of the discrete scheme at frozen decisions; the bar is
1e-5 relative per component (1e-4 against the oracle, whose F differs from
the GPU's only by rounding but is evaluated with its own root finder), also
at the benchmark's sharp kernel kappa = (64/pi)^2, one theta-bin wide.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import flux  # noqa: E402
from paper_2309_08655_gb300 import inputs as I  # noqa: E402
from paper_2309_08655_gb300 import rt  # noqa: E402

from . import gpu_util as G  # noqa: E402

KAPPA = 4.0
RTOL_FD = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available()


def _base():
    """The misaligned magnetar-like star (B0 = 1.6e14 G, P = 3.76 s, 30 deg,
    1.5 Msun, 11 km) at m_a = 1e-5 eV, rotation phase uniform per ray."""
    kw = I.stars_config1()[0]
    kw.update(m_a_eV=1e-5)
    return kw


def _p0(kw, incl=1.1):
    return torch.tensor([kw["m_a_eV"], kw["B0_G"], kw["theta_m"], kw["M_sun"], kw["R_km"], incl],
                        dtype=torch.float64)


def _steps(p):
    h = 1e-6 * np.abs(p.numpy())
    h[2] = h[5] = 1e-6
    return h


def _fd(fn, p, h):
    g = np.zeros(6)
    for k in range(6):
        e = torch.zeros(6, dtype=torch.float64)
        e[k] = h[k]
        g[k] = (fn(p + e) - fn(p - e)) / (2.0 * h[k])
    return g


def _oracle_F(oracle, base, p, u, kappa, rtol):
    """F by the oracle: its own sampling, trace and line-flux functional."""
    kw = dict(base)
    kw.update(m_a_eV=float(p[0]), B0_G=float(p[1]), theta_m=float(p[2]), M_sun=float(p[3]),
              R_km=float(p[4]))
    sv = oracle.star_vector(**kw)
    st, w, s = oracle.sample(sv, u)
    oracle.trace_forward(sv, oracle.trace_opts(rtol=rtol), st, s)
    return oracle.line_flux(sv, st, w, s, float(p[5]), kappa)


def test_adjoint_matches_finite_differences():
    kw = _base()
    n = 2048
    u = torch.from_numpy(I.sample_uniforms(4, n)).to(G.dev())
    p = _p0(kw).requires_grad_(True)
    F = flux.line_flux(p, kw, u, KAPPA)
    F.backward()
    g_adj = p.grad.numpy().copy()
    assert math.isfinite(float(F.detach())) and float(F.detach()) > 0

    def Fgpu(q):
        return float(flux.flux_forward(q, kw, u, KAPPA, rtol=RTOL_FD)[0].cpu()[0])

    pd = p.detach()
    g_fd = _fd(Fgpu, pd, _steps(pd))
    rel = np.abs(g_adj - g_fd) / np.maximum(np.abs(g_fd), 1e-300)
    assert np.all(np.isfinite(g_adj))
    assert np.all(rel < 1e-5), (g_adj, g_fd, rel)


def test_adjoint_replay_reproduces_forward_value():
    kw = _base()
    n = 1024
    u = torch.from_numpy(I.sample_uniforms(5, n)).to(G.dev())
    p = _p0(kw, incl=0.7)
    F, nacc, star, incl, opts = flux.flux_forward(p, kw, u, KAPPA)
    grad = torch.empty(6, dtype=torch.float64, device=G.dev())
    F2 = torch.empty(1, dtype=torch.float64, device=G.dev())
    ctr = torch.zeros(8, dtype=torch.int64, device=G.dev())
    nbytes = rt.rt_flux_gradient(star, n, u, nacc, incl, KAPPA, grad, F2, counters=ctr,
                                 opts=opts)
    torch.cuda.synchronize()
    # the same rays and steps; the functional is summed from per-ray terms that
    # the two kernels round differently (FMA contraction)
    assert abs(float(F2.cpu()[0]) - float(F.cpu()[0])) <= 1e-13 * abs(float(F.cpu()[0]))
    c = ctr.cpu().numpy()
    assert c[2] == n and c[4] == 0
    assert nbytes > 0


def test_adjoint_matches_oracle_reference_gradient(oracle):
    kw = _base()
    n = 512
    u_np = I.sample_uniforms(6, n)
    u = torch.from_numpy(u_np).to(G.dev())
    p = _p0(kw, incl=1.3).requires_grad_(True)
    F = flux.line_flux(p, kw, u, KAPPA)
    F.backward()
    g_adj = p.grad.numpy()
    pd = p.detach()
    F_or = _oracle_F(oracle, kw, pd.numpy(), u_np, KAPPA, 1e-10)
    assert abs(F_or - float(F.detach())) <= 1e-9 * abs(F_or)
    g_or = _fd(lambda q: _oracle_F(oracle, kw, q.numpy(), u_np, KAPPA, RTOL_FD), pd, _steps(pd))
    rel = np.abs(g_adj - g_or) / np.maximum(np.abs(g_or), 1e-300)
    assert np.all(rel < 1e-4), (g_adj, g_or, rel)


def test_gradient_rejects_unsupported_models():
    kw = _base()
    kw.update(plasma=4, plasma_a=8.0)      # the spherical test medium
    star = rt.Star(rt.make_params(**kw))
    n = 16
    u = torch.from_numpy(I.sample_uniforms(7, n)).to(G.dev())
    nacc = torch.zeros(n, dtype=torch.int32, device=G.dev())
    g = torch.empty(6, dtype=torch.float64, device=G.dev())
    F = torch.empty(1, dtype=torch.float64, device=G.dev())
    with pytest.raises(rt.RtError):
        rt.rt_flux_gradient(star, n, u, nacc, 1.0, KAPPA, g, F)


def test_mixed_sweep_close_to_fp64_sweep():
    """The mixed backward sweep (RT_PREC_MIXED: the adjoint of the state in
    FP64, the tangents of r_s, the omega_p^2 coefficient and the magnetic axis
    in FP32) over the same FP64 replay: the same F, and every gradient
    component within 1e-4 relative of the FP64 sweep's (FP32 rounding of the
    parameter products, summed over ~10^3 stages a ray; 1.3e-5 worst at the
    benchmark's 2^18 rays)."""
    kw = _base()
    n = 2048
    u = torch.from_numpy(I.sample_uniforms(4, n)).to(G.dev())
    g = {}
    for prec in ("fp64", "mixed"):
        p = _p0(kw).requires_grad_(True)
        F = flux.line_flux(p, kw, u, KAPPA, grad_precision=prec)
        F.backward()
        g[prec] = p.grad.numpy().copy()
    rel = np.abs(g["mixed"] - g["fp64"]) / np.abs(g["fp64"])
    assert np.all(np.isfinite(g["mixed"]))
    assert np.all(rel < 1e-4), (g, rel)
    # the replay (and so F) is FP64 in both
    F0, nacc, star, incl, _ = flux.flux_forward(_p0(kw), kw, u, KAPPA)
    grad = torch.empty(6, dtype=torch.float64, device=G.dev())
    F2 = torch.empty(1, dtype=torch.float64, device=G.dev())
    rt.rt_flux_gradient(star, n, u, nacc, incl, KAPPA, grad, F2,
                        opts=rt.make_opts(rtol=1e-10, precision=rt.PREC_MIXED))
    assert abs(float(F2.cpu()[0]) - float(F0.cpu()[0])) <= 1e-13 * abs(float(F0.cpu()[0]))


def test_line_flux_rejects_unknown_grad_precision():
    kw = _base()
    u = torch.from_numpy(I.sample_uniforms(4, 8)).to(G.dev())
    with pytest.raises(ValueError):
        flux.line_flux(_p0(kw), kw, u, KAPPA, grad_precision="fp16")


def test_adjoint_matches_oracle_at_the_benchmark_kappa(oracle):
    """The benchmark's functional: kappa = (64/pi)^2, a kernel one theta-bin
    (0.05 rad) wide, so each ray's term and its gradient vary 100 times
    faster with its end direction than at kappa = 4.  4096 rays toward
    inclination 1.1 rad (the benchmark's), oracle central differences at
    rtol 1e-12: 1e-4 per component."""
    kappa = (64.0 / math.pi) ** 2
    kw = _base()
    n = 4096
    u_np = I.sample_uniforms(8, n)
    u = torch.from_numpy(u_np).to(G.dev())
    p = _p0(kw, incl=1.1).requires_grad_(True)
    F = flux.line_flux(p, kw, u, kappa)
    F.backward()
    g_adj = p.grad.numpy()
    pd = p.detach()
    F_or = _oracle_F(oracle, kw, pd.numpy(), u_np, kappa, 1e-10)
    assert F_or > 0 and abs(F_or - float(F.detach())) <= 1e-8 * abs(F_or)
    g_or = _fd(lambda q: _oracle_F(oracle, kw, q.numpy(), u_np, kappa, RTOL_FD), pd, _steps(pd))
    rel = np.abs(g_adj - g_or) / np.maximum(np.abs(g_or), 1e-300)
    print("kappa = (64/pi)^2: adjoint", g_adj, "oracle FD", g_or, "rel", rel)
    assert np.all(rel < 1e-4), (g_adj, g_or, rel)


def _gradient(kw, u, prec, tape_max_bytes=-1, incl=1.1, kappa=KAPPA):
    """dF/dp through the C ABI with the sweep in `prec`; the store's bytes
    and the counters."""
    n = u.shape[1]
    F0, nacc, star, incl_r, _ = flux.flux_forward(_p0(kw, incl=incl), kw, u, kappa)
    grad = torch.empty(6, dtype=torch.float64, device=G.dev())
    F2 = torch.empty(1, dtype=torch.float64, device=G.dev())
    ctr = torch.zeros(8, dtype=torch.int64, device=G.dev())
    nbytes = rt.rt_flux_gradient(star, n, u, nacc, incl_r, kappa, grad, F2, counters=ctr,
                                 opts=rt.make_opts(rtol=1e-10, precision=prec),
                                 tape_max_bytes=tape_max_bytes)
    torch.cuda.synchronize()
    return (grad.cpu().numpy(), float(F2.cpu()[0]), float(F0.cpu()[0]), nbytes,
            ctr.cpu().numpy(), nacc)


def test_full_tape_and_checkpoints_give_the_same_gradient():
    """The full step tape (one replay) and the checkpointed recompute (a
    replay per segment more) take the same FP64 steps: the same F and
    gradient to rounding (the kernels contract multiply-adds differently, and
    a segment restarts from its checkpoint with the right-hand side
    re-evaluated; the sum over rays cancels, so a component can lose a few
    digits).  The tape's size is the documented 416 B per slot plus 488 B
    per ray."""
    kw = _base()
    n = 2048
    u = torch.from_numpy(I.sample_uniforms(9, n)).to(G.dev())
    gt, Ft, F0, bt, ct, nacc = _gradient(kw, u, rt.PREC_FP64)
    gc, Fc, _, bc, cc, _ = _gradient(kw, u, rt.PREC_FP64, tape_max_bytes=0)
    assert abs(Ft - Fc) <= 1e-14 * abs(Fc)
    assert abs(Ft - F0) <= 1e-13 * abs(F0)
    rel = np.abs(gt - gc) / np.abs(gc)
    assert np.all(rel < 1e-7), rel
    na = nacc.cpu().numpy().astype(np.int64)
    slots = na + na // 64 + 9
    assert bt == int(slots.sum()) * 416 + n * 488
    assert bc == int((na // 32 + 2).sum()) * 104
    # one replay against two: the first replay's attempts are counted by both
    assert ct[0] == cc[0] and ct[2] == cc[2] == n and ct[4] == cc[4] == 0


def test_full_tape_gradient_is_deterministic():
    """The longest-first order within a bucket follows the atomics; no ray's
    result depends on it and the sums run in index order: bit for bit."""
    kw = _base()
    u = torch.from_numpy(I.sample_uniforms(10, 3000)).to(G.dev())
    g1 = _gradient(kw, u, rt.PREC_FP64)[0]
    g2 = _gradient(kw, u, rt.PREC_FP64)[0]
    assert np.array_equal(g1, g2)


@pytest.mark.parametrize("store", ["tape", "checkpoints"])
def test_double_float_sweep_matches_fp64_sweep(store):
    """The double-float backward sweep (RT_PREC_DF; ~48-bit rounding on the
    FP32 pipe) over the same FP64 replay: within 1e-8 relative of the FP64
    sweep per component at the benchmark's kappa (the FP32 sweep's error is
    ~1e-4 there), and the same F (the replay is the same kernel)."""
    kappa = (64.0 / math.pi) ** 2
    kw = _base()
    u = torch.from_numpy(I.sample_uniforms(11, 4096)).to(G.dev())
    tmb = -1 if store == "tape" else 0
    g64, F64, _, _, _, _ = _gradient(kw, u, rt.PREC_FP64, tmb, kappa=kappa)
    gdf, Fdf, _, _, _, _ = _gradient(kw, u, rt.PREC_DF, tmb, kappa=kappa)
    assert F64 == Fdf
    rel = np.abs(gdf - g64) / np.abs(g64)
    assert np.all(rel < 1e-8), (g64, gdf, rel)
