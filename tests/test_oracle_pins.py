"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks one oracle function against something other than the oracle itself:
printed values of the paper (tests/golden/paper_values.txt), published known-answer
vectors (Philox), closed forms derived from the paper's definitions (moments, the
free-bead diffusion of Eq. 33, the simulated mobility tensor of Eqs. 40-41, the
periodic correction of Eq. 60), invariants (divergence-free wavelet field, Boltzmann
stationarity of one bead in a well), textbook routines (libm cos/sin, scipy quadrature
of the Fourier transform) and brute force written independently in numpy (energies).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O
from paper_1611_09160_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def params(**kw):
    p = dict(n_beads=2, box_L=64.0, lambda_min=2.0, lambda_max=32.0, A0=0.5, kT=1.0, bond_type=0, bond_k=0.0,
             bond_r0=2.0, fene_R0=3.0, wca_sigma=2.0, wca_eps=0.0, ext_kappa=0.0, planewave_mode=0, lcut=8,
             precision=0, seed=11, sim_id=0, colour_K=2, grid_f=16, n_cap=64, grid_layer=[0] * 16)
    p.update(kw)
    return p


def paper_value(name):
    for line in open(os.path.join(GOLD, "paper_values.txt")):
        if line.startswith(name + " "):
            f = line.split()
            return float(f[1]), float(f[2])
    raise KeyError(name)


# ---- test-side independent definitions -------------------------------------------------

def phitilde_np(k):
    """Eq. 25 (closed form); the test's own copy, valid for k >= 0.5."""
    k = np.asarray(k, dtype=float)
    return 4 * np.pi * (5 * k * np.sin(k) - (k ** 2 - 8) * np.cos(k) - 8) / k ** 6


def phitilde_by_quadrature(k):
    """Fourier transform of phi(r) = r^2/2 - r^3/3 - 1/6 on the unit ball (Eq. 24), by scipy."""
    f = lambda r: (r * r / 2 - r ** 3 / 3 - 1 / 6) * (np.sinc(k * r / np.pi)) * r * r
    return 4 * np.pi * integrate.quad(f, 0, 1, epsabs=1e-14, epsrel=1e-13)[0]


# ---- random numbers --------------------------------------------------------------------

def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = O.philox(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]
        n += 1
    assert n == 3


# ---- wavelet constants (Eqs. 22, 25, 42) ------------------------------------------------

def test_phitilde_series_and_closed_form():
    # value at 0 from the definition: 4 pi Int_0^1 phi r^2 dr = 4 pi (1/10 - 1/18 - 1/18) = -2 pi / 45
    assert O.phitilde(0.0) == pytest.approx(-2 * math.pi / 45, rel=1e-14)
    for k in [0.01, 0.3, 0.7, 1.5, 1.99, 2.0, 3.7, 10.0, 55.5]:
        assert O.phitilde(k) == pytest.approx(phitilde_by_quadrature(k), rel=1e-9, abs=1e-13)
    for k in [0.6, 1.0, 1.9]:   # series branch against the closed form where it does not cancel badly
        assert O.phitilde(k) == pytest.approx(float(phitilde_np(k)), rel=1e-9)


def test_moments_closed_forms_and_lambda_a():
    # derived: M4 = 8 pi^3/105, M6 = (2 pi)^3/5 (Parseval), M3 = (16 pi^2/105)(9/8 - ln 2)
    assert O.moment(4) == pytest.approx(8 * math.pi ** 3 / 105, rel=1e-10)
    assert O.moment(6) == pytest.approx((2 * math.pi) ** 3 / 5, rel=1e-9)
    M3 = O.moment(3)
    assert M3 == pytest.approx(16 * math.pi ** 2 / 105 * (9 / 8 - math.log(2)), rel=1e-10)
    la = 2 / math.pi * O.moment(4) / M3            # Eq. 42
    v, tol = paper_value("lambda_a")
    assert la == pytest.approx(v, rel=tol)
    assert O.lambda_a() == pytest.approx(la, rel=1e-10)
    lm, _ = paper_value("lambda_min_bar")
    a, tol = paper_value("a_bar")
    assert lm / O.lambda_a() == pytest.approx(a, rel=tol)


def test_G_tail_integral():
    # G(0) = M3; G decreasing; large-Q asymptote 2 pi^2 Q^-4 (phi~^2 ~ 16 pi^2 k^-8 cos^2 k)
    g = O.G([0.0, 1.0, 5.0, 40.0, 400.0])
    assert g[0] == pytest.approx(16 * math.pi ** 2 / 105 * (9 / 8 - math.log(2)), rel=1e-10)
    assert np.all(np.diff(g) < 0)
    assert g[4] == pytest.approx(2 * math.pi ** 2 * 400.0 ** -4, rel=1e-2)   # oscillating part is O(1/Q)
    # against scipy on a finite range plus the same asymptote
    q = 3.0
    f = lambda x: x ** 3 * phitilde_np(x) ** 2
    edges = np.arange(q, 2000.0, math.pi / 2)
    ref = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-12)[0] for a, b in zip(edges[:-1], edges[1:]))
    ref += 2 * math.pi ** 2 * edges[-1] ** -4
    assert O.G([q])[0] == pytest.approx(ref, rel=1e-7)


# ---- own elementary functions ----------------------------------------------------------

def test_own_cos_sin_and_cube_root():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    t = np.concatenate([np.linspace(0, 1, 2001), np.random.default_rng(1).random(2000) * 7 - 3])
    c = np.array([O.cos2pi(x) for x in t])
    s = np.array([O.sin2pi(x) for x in t])
    c_ref = np.array([float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(x)))) for x in t])
    s_ref = np.array([float(mpmath.sin(2 * mpmath.pi * mpmath.mpf(float(x)))) for x in t])
    assert np.max(np.abs(c - c_ref)) < 2.3e-16
    assert np.max(np.abs(s - s_ref)) < 2.3e-16
    cf = np.array([O.cos2pi_f(x) for x in t[:2000]])
    assert np.max(np.abs(cf - np.cos(2 * np.pi * t[:2000]))) < 3e-7
    for lo, hi in [(2.0, 4.0), (64.0, 102.4), (2.0, 2.5)]:
        for u in [0.0, 0.3, 0.999999]:
            w = lo ** -3 - u * (lo ** -3 - hi ** -3)
            assert O.inv_cbrt(w, lo) == pytest.approx(w ** (-1 / 3), rel=2e-15)


# ---- the wavelet field (Eqs. 21, 23, 24; Appendix D) ------------------------------------

def test_wavelet_field_properties():
    o = O.Oracle(params(), np.array([[10.0, 10, 10], [20, 20, 20]]), np.array([1, 1], np.int32))
    rng = np.random.default_rng(3)
    b = np.array([30.0, 31.0, 29.5])
    lam, Aw = 5.0, 0.7
    for _ in range(20):
        p = rng.normal(size=3)
        p /= np.linalg.norm(p)
        x = rng.normal(size=3)
        x *= rng.random() * 0.9 / np.linalg.norm(x)
        pt = b + lam * x
        d = o.wavelet_field(b, lam, p, Aw, pt)
        # transverse: delta . x = 0; magnitude A_w (1 - |x|) |p x x|
        assert abs(d @ x) < 1e-13
        assert np.linalg.norm(d) == pytest.approx(Aw * (1 - np.linalg.norm(x)) * np.linalg.norm(np.cross(p, x)), rel=1e-12)
        # divergence-free (Eq. 17) by central differences
        h = 1e-4
        div = sum((o.wavelet_field(b, lam, p, Aw, pt + h * e)[a] - o.wavelet_field(b, lam, p, Aw, pt - h * e)[a]) / (2 * h)
                  for a, e in enumerate(np.eye(3)))
        assert abs(div) < 1e-8
    # Eq. 23 for p = z:  w = r sin(theta) (1 - r) phi_hat
    p = np.array([0.0, 0.0, 1.0])
    x = np.array([0.3, -0.2, 0.4])
    r = np.linalg.norm(x)
    phi_hat = np.array([-x[1], x[0], 0.0]) / math.hypot(x[0], x[1])
    sin_t = math.hypot(x[0], x[1]) / r
    want = Aw * r * sin_t * (1 - r) * phi_hat
    assert np.allclose(o.wavelet_field(b, lam, p, Aw, b + lam * x), want, rtol=1e-12, atol=1e-14)
    # zero on and outside the support (Eq. 16)
    assert np.all(o.wavelet_field(b, lam, p, Aw, b + np.array([lam, 0, 0])) == 0)
    assert np.all(o.wavelet_field(b, lam, p, Aw, b + np.array([0, 1.01 * lam, 0])) == 0)


# ---- energies: oracle dU against an independent numpy brute force ----------------------

def energy_np(pos, chain_len, L, p):
    """Total energy: WCA (Eq. 2) on all pairs, bonds on chain neighbours, external well."""
    n = len(pos)
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    r2 = np.sum(d * d, axis=-1)
    iu = np.triu_indices(n, 1)
    r2p = r2[iu]
    E = 0.0
    if p["wca_eps"]:
        rc2 = (2 ** (1 / 6) * p["wca_sigma"]) ** 2
        m = r2p < rc2
        s6 = (p["wca_sigma"] ** 2 / r2p[m]) ** 3
        E += np.sum(4 * p["wca_eps"] * (s6 * s6 - s6) + p["wca_eps"])
    ends = np.cumsum(chain_len)
    bonded = np.ones(n - 1, bool)
    bonded[ends[:-1] - 1] = False
    rb = np.sqrt(r2[np.arange(n - 1), np.arange(1, n)])[bonded]
    if p["bond_type"] == 1:
        E += np.sum(0.5 * p["bond_k"] * (rb - p["bond_r0"]) ** 2)
    elif p["bond_type"] == 2:
        x = (rb / p["fene_R0"]) ** 2
        E += np.inf if np.any(x >= 1) else np.sum(-0.5 * p["bond_k"] * p["fene_R0"] ** 2 * np.log(1 - x))
    if p["ext_kappa"]:
        c = pos - L / 2
        c -= L * np.round(c / L)
        E += 0.5 * p["ext_kappa"] * np.sum(c * c)
    return E


@pytest.mark.parametrize("bond_type", [1, 2])
def test_delta_u_matches_brute_force(bond_type):
    sysm = I.make_system([12, 9, 1, 1], 0, 14.0, seed=5)   # small box: many pairs, chains across the boundary
    p = params(n_beads=sysm.n_beads, box_L=14.0, lambda_max=7.0, bond_type=bond_type, bond_k=30.0, bond_r0=2.0,
               fene_R0=3.2, wca_eps=1.0, ext_kappa=0.05)
    o = O.Oracle(p, sysm.pos, sysm.chain_len)
    E0 = energy_np(sysm.pos, sysm.chain_len, 14.0, p)
    assert o.total_energy() == pytest.approx(E0, rel=1e-12)
    rng = np.random.default_rng(8)
    for trial in range(40):
        k = rng.integers(1, 8)
        ids = np.sort(rng.choice(sysm.n_beads, size=k, replace=False))
        newp = sysm.pos[ids] + rng.normal(scale=0.15, size=(k, 3))
        newp %= 14.0
        after = sysm.pos.copy()
        after[ids] = newp
        want = energy_np(after, sysm.chain_len, 14.0, p) - E0
        got = o.delta_u(ids, newp)
        if np.isinf(want):
            assert np.isinf(got) and got > 0
        else:
            assert got == pytest.approx(want, rel=1e-9, abs=1e-9)


# ---- sampling distributions (Eqs. 26, 32; Appendix D) ----------------------------------

def test_layers_partition_P_lambda():
    o = O.Oracle(params(box_L=409.5, lambda_max=204.75), np.array([[1.0, 1, 1], [5, 5, 5]]), np.array([1, 1], np.int32))
    lo, hi, mass, expect = o.layers()
    assert len(lo) == 7 and lo[0] == 2.0 and hi[-1] == 204.75
    assert np.all(hi[:-1] == lo[1:])
    assert mass.sum() == pytest.approx(1.0, rel=1e-14)
    Nl = 3 / (2.0 ** -3 - 204.75 ** -3)         # Eq. 32
    for a, b, m in zip(lo, hi, mass):
        assert m == pytest.approx(integrate.quad(lambda x: Nl * x ** -4, a, b)[0], rel=1e-10)


def test_lambda_within_band_follows_P_lambda():
    o = O.Oracle(params(box_L=409.5, lambda_max=204.75), np.array([[1.0, 1, 1], [5, 5, 5]]), np.array([1, 1], np.int32))
    lo, hi, _, _ = o.layers()
    for l in [0, 3, 6]:
        lam, bead = o.sample_slots(l, 20000)
        a, b = lo[l], hi[l]
        cdf = lambda x: (a ** -3 - np.asarray(x) ** -3) / (a ** -3 - b ** -3)
        assert stats.kstest(lam, cdf).pvalue > 1e-3
        assert np.all((lam >= a) & (lam <= b))
        assert set(np.unique(bead)) == {0, 1}


def test_ball_points_and_polarisation():
    o = O.Oracle(params(), np.array([[1.0, 1, 1], [5, 5, 5]]), np.array([1, 1], np.int32))
    V = o.sample_ball(3, 40000)
    r = np.linalg.norm(V, axis=1)
    assert np.all(r <= 1.0)
    assert stats.kstest(r, lambda x: np.clip(x, 0, 1) ** 3).pvalue > 1e-3     # uniform in the ball
    assert np.all(np.abs(V.mean(0)) < 4 * np.sqrt(0.2 / len(V)))
    P = o.sample_polarisation(4, 40000)
    assert np.allclose(np.linalg.norm(P, axis=1), 1.0, atol=1e-15)
    assert np.allclose(P.T @ P / len(P), np.eye(3) / 3, atol=0.012)              # isotropic
    assert stats.kstest(P[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3         # Archimedes: z uniform


# ---- dynamics pins ---------------------------------------------------------------------

def _msd_per_move(o, sweeps, batches):
    x0 = o.positions(unwrapped=True)
    acc0 = o.stats().accepted_total
    per = []
    for _ in range(batches):
        o.sweep(sweeps)
        x1 = o.positions(unwrapped=True)
        acc1 = o.stats().accepted_total
        per.append(np.mean(np.sum((x1 - x0) ** 2, axis=1)) / (acc1 - acc0))
        x0, acc0 = x1, acc1
    per = np.array(per)
    return per.mean(), per.std(ddof=1) / np.sqrt(len(per))


@pytest.mark.parametrize("centring", [0, 1])
def test_free_bead_diffusion_wavelets(centring):
    """Eq. 33: per move <dr^2> = (2/105) A0^2 N_lambda (1/lmin - 1/lmax) / N for any
    configuration of non-interacting beads, and MSD = a^2 t (Eq. 34, a = lmin/lambda_a). With the
    centre uniform in the box (Sec. V.D) and A_w from the mean count the same holds: P_b A_w^2 is
    3 A0^2 / (4 pi N lambda) in both schemes."""
    N, L = 24, 64.0
    s = I.make_system([], N, L, seed=2)
    p = params(n_beads=N, box_L=L, seed=21, centring=centring)
    o = O.Oracle(p, s.pos, s.chain_len)
    m, se = _msd_per_move(o, 200, 30)
    Nl = 3 / (2.0 ** -3 - 32.0 ** -3)
    want = 2 / 105 * 0.25 * Nl * (1 / 2.0 - 1 / 32.0) / N
    assert abs(m - want) < 4 * se + 1e-3 * want
    st = o.stats()
    assert st.accepted_total == sum(st.attempts)                 # nothing rejects without interactions
    a = 2.0 / O.lambda_a()
    assert st.dt_move * a * a == pytest.approx(want, rel=1e-12)


def test_free_bead_diffusion_with_plane_waves():
    """Wavelets + periodic plane waves: per move (1-P_F)<dr^2>_w + P_F sum_k P(k) A_F(k)^2/2,
    predicted from the mode tables; and the infinite-system identity of Eq. 57."""
    N, L = 8, 24.0
    s = I.make_system([], N, L, seed=4)
    p = params(n_beads=N, box_L=L, lambda_max=12.0, planewave_mode=1, lcut=8, seed=5, grid_f=8)
    o = O.Oracle(p, s.pos, s.chain_len)
    modes, prob, R, PF = o.pw_modes()
    l2 = np.sum(modes.astype(float) ** 2, axis=1)
    nz = l2 > 0
    drF = np.sum(prob[nz] * 4 * 0.25 / ((2 * np.pi / L) ** 2 * l2[nz] * 5 * N) / 2)
    Nl = 3 / (2.0 ** -3 - 12.0 ** -3)
    drw = 2 / 105 * 0.25 * Nl * (1 / 2.0 - 1 / 12.0) / N
    want = (1 - PF) * drw + PF * drF
    m, se = _msd_per_move(o, 400, 30)
    assert abs(m - want) < 4 * se + 2e-3 * want
    assert o.stats().pw_attempts > 20
    # infinite system: (1 - P_F)<dr^2>_w + P_F <dr^2>_F = 6 A0^2 lmin^2 / (105 N)  (Eqs. 53, 54, 57)
    PFi = (2.0 / 12.0) ** 3
    drFi = 6 * 0.25 * 12.0 ** 2 / (105 * N)
    assert (1 - PFi) * drw + PFi * drFi == pytest.approx(6 * 0.25 * 4 / (105 * N), rel=1e-13)


def Ow(r, lp, A0):
    """Eq. 40: (g_rr, g_tt) of O_w(r; lambda', infinity), by scipy quadrature."""
    def f(q, which):
        Q = q * r / lp
        ph = float(phitilde_np(q)) if q >= 0.5 else O.phitilde(q)
        si = special.sici(Q)[0]
        b = (math.sin(Q) - Q * math.cos(Q)) / Q ** 2
        return q ** 3 * ph ** 2 * ((2 * si - 2 * b) if which == "rr" else (si + b))
    pts = np.arange(0, 400, math.pi)
    out = []
    for w in ("rr", "tt"):
        tot = sum(integrate.quad(f, a, b, args=(w,), limit=200)[0] for a, b in zip(pts[:-1], pts[1:]))
        out.append(A0 ** 2 / (3 * math.pi * r) * tot)
    return np.array(out)


@pytest.mark.parametrize("r,centring,L,batches", [(3.0, 0, 200.0, 10), (12.0, 0, 200.0, 10), (12.0, 1, 64.0, 40)])
def test_two_bead_correlations_follow_Ow(r, centring, L, batches):
    """<dr_0 (x) dr_1> per proposal = 3 N_lambda/(16 pi^2 N) O_w(r; lmin, lmax)  (Eqs. 39-41;
    the constant follows from the Fourier transform of the proposal average). Also close to
    Rotne-Prager (Eqs. 11-12) at a = lmin/lambda_a between lmin and lmax (Sec. V.D: "very close")."""
    A0, lmin, lmax = 0.5, 2.0, 32.0
    pos = np.array([[L / 2, L / 2, L / 2], [L / 2 + r, L / 2, L / 2]])
    o = O.Oracle(params(box_L=L, lambda_max=lmax, seed=17, centring=centring), pos, np.array([1, 1], np.int32))
    est = []
    for b in range(batches):
        c01, c00, _ = o.propose_moments(100000, offset=b * 100000)
        est.append([c01[0, 0], c01[1, 1], np.trace(c00)])
    est = np.array(est)
    m, se = est.mean(0), est.std(0, ddof=1) / np.sqrt(len(est))
    Nl = 3 / (lmin ** -3 - lmax ** -3)
    c = 3 * Nl / (16 * math.pi ** 2 * 2)
    want = c * (Ow(r, lmin, A0) - Ow(r, lmax, A0))
    assert abs(m[0] - want[0]) < 4.5 * se[0]
    assert abs(m[1] - want[1]) < 4.5 * se[1]
    tr0 = 4 * A0 ** 2 * (8 * math.pi ** 3 / 105) / (3 * math.pi) * (1 / lmin - 1 / lmax)
    assert abs(m[2] - c * tr0) < 4.5 * se[2]
    # Rotne-Prager (Eqs. 11-12), normalised by the self mobility 1/(6 pi eta a): compare the
    # measured tensor plus the part lambda > lmax (which plane waves supply, Sec. VI), i.e.
    # the full O_w(r; lmin, infinity) of Sec. V.D, with a = lmin / lambda_a.
    if centring:
        return                   # the uniform-centre scheme: pinned against O_w above (noisier estimate)
    a = lmin / O.lambda_a()
    rp_rr = 6 * math.pi * a * (2 / (8 * math.pi * r) - 2 / (12 * math.pi * r) * (a / r) ** 2)
    rp_tt = 6 * math.pi * a * (1 / (8 * math.pi * r) + 1 / (12 * math.pi * r) * (a / r) ** 2)
    tail = c * Ow(r, lmax, A0)
    self_ = (m[2] + c * 4 * A0 ** 2 * (8 * math.pi ** 3 / 105) / (3 * math.pi * lmax)) / 3
    assert (m[0] + tail[0]) / self_ == pytest.approx(rp_rr, rel=0.08)
    assert (m[1] + tail[1]) / self_ == pytest.approx(rp_tt, rel=0.08)


@pytest.mark.parametrize("acceptance,centring", [(0, 0), (1, 0), (0, 1)])
def test_boltzmann_one_bead_in_a_well(acceptance, centring):
    """One bead in a harmonic well with wavelet moves: the proposal is symmetric and position
    independent (centre near the bead or uniform in the box), so Metropolis (Eq. 20) and Glauber
    acceptance both leave exp(-U/kT) invariant exactly."""
    kappa, kT = 0.3, 1.0
    # a uniform centre hits the lone bead only when the ball covers it: a smaller box, and an
    # amplitude that keeps A_w = A0 lam / sqrt(nbar) near the well's width
    L, lmax, A0, sweeps = (16.0, 8.0, 0.2, 2_000_000) if centring else (64.0, 16.0, 0.5, 400_000)
    p = params(n_beads=1, box_L=L, lambda_max=lmax, ext_kappa=kappa, kT=kT, seed=99, acceptance=acceptance,
               centring=centring, A0=A0)
    o = O.Oracle(p, np.array([[L / 2, L / 2, L / 2]]), np.array([1], np.int32))
    o.sweep(2000)
    x = o.sweep_record(sweeps) - L / 2
    bm = x.reshape(200, -1, 3)
    var_b = np.mean(bm ** 2, axis=1)                  # batch means of x^2
    v, se = var_b.mean(0), var_b.std(0, ddof=1) / np.sqrt(len(var_b))
    assert np.all(np.abs(v - kT / kappa) < 4.5 * se + 0.01 * kT / kappa)
    if centring:
        return               # the lone bead moves in ~3% of the sweeps: too few tail visits for a histogram
    # histogram of x against the Gaussian: bin frequencies as batch means (the samples of a chain
    # are correlated over hundreds of sweeps, so each bin is tested against its batch spread)
    edges = np.concatenate([[-np.inf], np.linspace(-2.5, 2.5, 11) * math.sqrt(kT / kappa), [np.inf]])
    pr = np.diff(stats.norm.cdf(edges / math.sqrt(kT / kappa)))
    freq = np.array([np.histogram(b[:, 0], bins=edges)[0] / len(b) for b in bm])
    f, se = freq.mean(0), freq.std(0, ddof=1) / math.sqrt(len(freq))
    assert np.all(np.abs(f - pr) < 4.5 * se + 2e-3)


@pytest.mark.parametrize("L", [40.0, 80.0, 160.0])
def test_periodic_mobility_finite_box(L):
    """Eq. 60: the periodic self-mobility is the infinite one times (1 - 2.837 a/L), with
    a = lmin/lambda_a. From the oracle's mode tables and P_F (Eqs. 48, 51, 55, 56)."""
    A0, lmin = 0.5, 2.0
    o = O.Oracle(params(n_beads=1, box_L=L, lambda_max=L / 2, planewave_mode=1, lcut=15, grid_f=8),
                 np.array([[1.0, 1, 1]]), np.array([1], np.int32))
    modes, prob, R, PF = o.pw_modes()
    l2 = np.sum(modes.astype(float) ** 2, axis=1)
    nz = l2 > 0
    drF = np.sum(prob[nz] * 4 * A0 ** 2 / ((2 * np.pi / L) ** 2 * l2[nz] * 5) / 2)
    Nl = 3 / (lmin ** -3 - (L / 2) ** -3)
    drw = 2 / 105 * A0 ** 2 * Nl * (1 / lmin - 2 / L)
    ratio = ((1 - PF) * drw + PF * drF) / (6 * A0 ** 2 * lmin ** 2 / 105)
    a = lmin / O.lambda_a()
    assert ratio == pytest.approx(1 - 2.837 * a / L, abs=4e-5)


def test_plane_wave_normalisation_converges():
    """R -> 1 as the mode set grows at lambda_max = L/2 (continuum limit of Eq. 55), and the
    k = 0 mode carries 0.1018 of the probability at |l| <= 8."""
    Rs = []
    for lcut in (4, 8, 16, 32):
        o = O.Oracle(params(n_beads=1, planewave_mode=1, lcut=lcut), np.array([[1.0, 1, 1]]), np.array([1], np.int32))
        modes, prob, R, PF = o.pw_modes()
        Rs.append(R)
        n_expected = sum(1 for x in range(-lcut, lcut + 1) for y in range(-lcut, lcut + 1)
                         for z in range(-lcut, lcut + 1) if x * x + y * y + z * z <= lcut * lcut)
        assert len(modes) == n_expected
        assert prob.sum() == pytest.approx(1.0, rel=1e-13)
        if lcut == 8:
            assert prob[np.all(modes == 0, axis=1)][0] == pytest.approx(0.1018, abs=1e-4)
            assert PF == pytest.approx(1 / (1 + R * (16.0 ** 3 - 1)), rel=1e-14)
    Rs = np.array(Rs)
    assert np.all(np.diff(Rs) < 0) and np.all(Rs > 1)
    assert (Rs[3] - 1) < 0.55 * (Rs[2] - 1)          # roughly 1/lcut convergence


def test_metropolis_rejects_overstretched_fene_and_counts():
    # a two-bead FENE chain close to R0: large moves overstretch and must reject
    p = params(n_beads=2, box_L=64.0, lambda_max=32.0, bond_type=2, bond_k=30.0, fene_R0=2.05, wca_eps=1.0, seed=3,
               A0=2.0)
    o = O.Oracle(p, np.array([[30.0, 30, 30], [32.0, 30, 30]]), np.array([2], np.int32))
    o.sweep(3000)
    x = o.positions(unwrapped=True)
    assert np.linalg.norm(x[1] - x[0]) < 2.05
    st = o.stats()
    assert 0 < sum(st.accepts) < sum(st.attempts)


def test_coloured_schedule_keeps_free_diffusion_and_defers_correctly():
    """The colouring only reorders moves: free-bead diffusion per move still follows Eq. 33.
    With coarse cells too small for the support every concurrent attempt is deferred."""
    from paper_1611_09160_gb300 import schedule
    N = 400
    s = I.free_spheres(N, 2e-3, seed=9)
    L = s.box_L
    sch = schedule.choose(L, 2.0, L / 2, 0.5, 2.0, 0.0)
    assert sch["grid_layer"][0] > 0
    p = params(n_beads=N, box_L=L, lambda_max=L / 2, seed=31, **sch)
    o = O.Oracle(p, s.pos, s.chain_len)
    m, se = _msd_per_move(o, 20, 20)
    lo, hi, _, _ = o.layers()
    Nl = 3 / (2.0 ** -3 - (L / 2) ** -3)
    want = 2 / 105 * 0.25 * Nl * (1 / 2.0 - 2 / L) / N
    assert abs(m - want) < 4 * se + 1e-3 * want
    st = o.stats()
    assert sum(st.attempts) == sum(st.accepts)
    # tiny coarse cells: every concurrent attempt of layer 0 must be deferred
    # region side 2h below the smallest influence diameter 2 * 1.125 * lambda_min = 4.5
    G = 2 * int(math.ceil(L / 2.2 / 2))
    assert 2 * L / G < 4.5
    fine = dict(sch, grid_layer=[G] + [0] * 15)
    o2 = O.Oracle(params(n_beads=N, box_L=L, lambda_max=L / 2, seed=31, **fine), s.pos, s.chain_len)
    o2.sweep(1)
    st2 = o2.stats()
    assert st2.deferred[0] == st2.attempts[0] > 0
    out, n = o2.trace_layer(0)
    assert np.all(out & 4)
    # second-level colouring: regions on a grid of K floor(G / 2K) cells per axis are about twice
    # as wide, so some of the same deferred slots now fit; the rest run serially (flags 4 | 8);
    # every slot is still attempted once and the run equals the serial order's statistics
    p3 = params(n_beads=N, box_L=L, lambda_max=L / 2, seed=31, **dict(fine, level2=1))
    o3 = O.Oracle(p3, s.pos, s.chain_len)
    o3.sweep(1)
    st3 = o3.stats()
    assert st3.attempts[0] == st2.attempts[0] and st3.deferred[0] == st3.attempts[0]
    out3, n3 = o3.trace_layer(0)
    assert np.all(out3 & 4)
    lvl2 = (out3 & 8) == 0
    assert 0 < lvl2.sum() < len(out3)
    assert np.all(n3[lvl2] <= 256)
    # level 2 never applies to a grid without two second-level cells per colour and axis
    o4 = O.Oracle(params(n_beads=N, box_L=L, lambda_max=L / 2, seed=31,
                         **dict(sch, grid_layer=[6] + [0] * 15, level2=1)), s.pos, s.chain_len)
    o4.sweep(1)
    assert not np.any(o4.trace_layer(0)[0] & 8)
    # nor to a layer whose bit the mask leaves out
    o6 = O.Oracle(params(n_beads=N, box_L=L, lambda_max=L / 2, seed=31, **dict(fine, level2=0xfffe)), s.pos, s.chain_len)
    o6.sweep(1)
    assert np.array_equal(o6.trace_layer(0)[0], out)
    # the schedule with the second level keeps Eq. 33
    o5 = O.Oracle(params(n_beads=N, box_L=L, lambda_max=L / 2, seed=37, **dict(fine, level2=1)), s.pos, s.chain_len)
    m5, se5 = _msd_per_move(o5, 20, 20)
    assert abs(m5 - want) < 4 * se5 + 1e-3 * want


# ---- plane-wave polarisation, field and recycling (Sec. VI; Appendix D) -----------------

def test_plane_wave_polarisation_is_transverse_unit_and_uniform():
    """Appendix D: e is a unit vector perpendicular to k, at a uniform angle about k; then
    <e (x) e> over the angle is (1 - k^ (x) k^)/2, the identity Sec. VI uses to turn the
    Fourier-space tensor into an expectation over e."""
    o = O.Oracle(params(n_beads=1, planewave_mode=1, lcut=8), np.array([[1.0, 1, 1]]), np.array([1], np.int32))
    modes, _, _, _ = o.pw_modes()
    psis = (np.arange(64) + 0.5) / 64            # a uniform grid of angles (in turns)
    for l in modes:
        if not np.any(l):
            continue
        kh = l / np.linalg.norm(l)
        E = np.array([O.pw_polarisation(l, s) for s in psis])
        assert np.allclose(np.linalg.norm(E, axis=1), 1.0, atol=2e-15)
        assert np.max(np.abs(E @ kh)) < 2e-15
        assert np.allclose(E.T @ E / len(E), (np.eye(3) - np.outer(kh, kh)) / 2, atol=1e-14)
    # the angle turns e about k: a quarter turn gives an orthogonal vector, half a turn -e
    l = np.array([2, -1, 3], np.int32)
    e0, e1, e2 = (O.pw_polarisation(l, s) for s in (0.1, 0.35, 0.6))
    assert abs(e0 @ e1) < 1e-15 and np.allclose(e2, -e0, atol=1e-15)


def test_plane_wave_field_divergence_free_periodic_and_amplitude():
    """Eq. 47 with the amplitude of Eq. 48: delta = A_F cos(k.r + Phi) e is transverse to k,
    divergence-free (central differences), periodic in the box (k commensurate), and its
    largest magnitude over the phase is A_F = 2 A0 / (k sqrt(5 N)) (dU_est/mu = A0^2 M6/(2 pi)^3,
    M6/(2 pi)^3 = 1/5)."""
    L, N, A0 = 24.0, 7, 0.6
    s = I.make_system([], N, L, seed=3)
    o = O.Oracle(params(n_beads=N, box_L=L, lambda_max=12.0, A0=A0, planewave_mode=1, lcut=8, grid_f=8),
                 s.pos, s.chain_len)
    rng = np.random.default_rng(5)
    for l in [(1, 0, 0), (0, 0, 2), (1, -2, 3), (4, 4, -1)]:
        l = np.array(l, np.int32)
        k = 2 * np.pi * l / L
        AF = 2 * A0 / (np.linalg.norm(k) * math.sqrt(5 * N))
        for _ in range(5):
            phi, psi = rng.random(), rng.random()
            pt = rng.random(3) * L
            d = o.planewave_field(l, phi, psi, pt)
            assert abs(d @ k) < 1e-13
            h = 1e-5
            div = sum((o.planewave_field(l, phi, psi, pt + h * e)[a] - o.planewave_field(l, phi, psi, pt - h * e)[a])
                      / (2 * h) for a, e in enumerate(np.eye(3)))
            assert abs(div) < 1e-8
            for a in range(3):
                shifted = pt.copy()
                shifted[a] += L
                assert np.allclose(o.planewave_field(l, phi, psi, shifted), d, atol=1e-12)
        # over the phase, |delta| reaches A_F (at k.r + Phi = 0) and never exceeds it
        pt = np.array([1.0, 2.0, 3.0])
        phase0 = (l @ pt) / L
        mags = [np.linalg.norm(o.planewave_field(l, ph, 0.3, pt)) for ph in np.linspace(0, 1, 101)]
        assert max(mags) <= AF * (1 + 1e-14)
        assert np.linalg.norm(o.planewave_field(l, -phase0, 0.3, pt)) == pytest.approx(AF, rel=1e-13)


def _signed_perm(a, b):
    """(permutation, signs) taking the components of a to those of b, when the three absolute
    components of a are distinct (so the order is identified); a sign is None for a zero
    component. None when the order cannot be identified."""
    aa = np.abs(a)
    if len(set(aa.tolist())) < 3:
        return None
    if sorted(np.abs(b).tolist()) != sorted(aa.tolist()):
        return None
    perm = tuple(int(np.where(aa == abs(x))[0][0]) for x in b)
    signs = tuple(None if x == 0 else int(np.sign(x) != np.sign(a[p])) for x, p in zip(b, perm))
    return perm, signs


def test_plane_wave_recycling_of_k():
    """Appendix D, parameter recycling: after a rejected periodic plane wave the next one keeps
    |k| by permuting the components (each of the six orders equally likely) and flipping each
    sign with probability 1/2; after an acceptance the next mode is drawn afresh."""
    L, N = 12.0, 40
    s = I.make_system([N], 0, L, seed=7)       # one dense chain: large plane waves reject often
    p = params(n_beads=N, box_L=L, lambda_max=6.0, A0=0.35, bond_type=1, bond_k=100.0, wca_eps=1.0,
               planewave_mode=1, lcut=8, grid_f=5, seed=23)
    o = O.Oracle(p, s.pos, s.chain_len)
    o.planewave(60000)
    out, packed = o.trace_pw()
    assert len(out) == 60000
    lv = np.stack([(packed & 0xFF) - 128, ((packed >> 8) & 0xFF) - 128, ((packed >> 16) & 0xFF) - 128], axis=1)
    rej = np.where(out[:-1] == 2)[0]
    acc = np.where(out[:-1] == 1)[0]
    assert len(rej) > 5000 and len(acc) > 5000
    # every rejection: the next wave vector has the same components up to order and sign
    same = np.sort(np.abs(lv[rej]), axis=1) == np.sort(np.abs(lv[rej + 1]), axis=1)
    assert np.all(same)
    # uniform over the 6 orders and the 8 sign patterns, independently
    counts_p, counts_s = {}, np.zeros((3, 2))
    for m in rej:
        r = _signed_perm(lv[m], lv[m + 1])
        if r is None:
            continue
        counts_p[r[0]] = counts_p.get(r[0], 0) + 1
        for a in range(3):
            if r[1][a] is not None:
                counts_s[a, r[1][a]] += 1
    cp = np.array(list(counts_p.values()))
    assert len(cp) == 6 and cp.sum() > 1500
    assert stats.chisquare(cp).pvalue > 1e-4
    for a in range(3):
        assert stats.binomtest(int(counts_s[a, 1]), int(counts_s[a].sum()), 0.5).pvalue > 1e-4
    # after an acceptance the carry is cleared: the next mode is a signed permutation of the
    # previous one only as often as a fresh draw from P(k_l) lands on one
    modes, prob, _, _ = o.pw_modes()
    key = {tuple(m): q for m, q in zip(modes.tolist(), prob)}
    cls = {}
    for m, q in zip(modes.tolist(), prob):
        c = tuple(sorted(abs(x) for x in m))
        cls[c] = cls.get(c, 0.0) + q
    expect = sum(cls[tuple(sorted(abs(int(x)) for x in lv[m]))] for m in acc)
    seen = int(np.sum(np.all(np.sort(np.abs(lv[acc]), axis=1) == np.sort(np.abs(lv[acc + 1]), axis=1), axis=1)))
    assert abs(seen - expect) < 5 * math.sqrt(expect) + 5
    assert seen < 0.6 * len(acc)
    assert key[(0, 0, 0)] > 0


def test_boltzmann_one_bead_in_a_well_with_plane_waves():
    """One bead in a harmonic well moved by periodic plane waves only, with an amplitude large
    enough that about half of them reject, so the |k| carry is in play. For a fixed wave vector
    the displacement A_F cos(theta) e with theta uniform is symmetric and position-independent,
    so each move leaves exp(-U/kT) invariant (Eq. 20); the variance must be kT/kappa."""
    kappa, kT = 0.3, 1.0
    p = params(n_beads=1, box_L=24.0, lambda_max=12.0, A0=2.0, ext_kappa=kappa, kT=kT, planewave_mode=1, lcut=8,
               grid_f=8, seed=71)
    o = O.Oracle(p, np.array([[12.0, 12.0, 12.0]]), np.array([1], np.int32))
    o.planewave(2000)
    xs, nacc, ntot = [], 0, 0
    for _ in range(10000):
        o.planewave(250)
        out, _ = o.trace_pw()
        nacc += int(np.sum(out == 1))
        ntot += len(out)
        xs.append(o.positions()[0] - 12.0)
    xs = np.array(xs)
    assert 0.3 < nacc / ntot < 0.6
    v, se = np.mean(xs ** 2, axis=0), np.std(xs ** 2, axis=0) / np.sqrt(len(xs))
    assert np.all(np.abs(v - kT / kappa) < 4.5 * se + 0.01 * kT / kappa)
    edges = np.linspace(-3, 3, 13) * math.sqrt(kT / kappa)
    h, _ = np.histogram(xs[:, 0], bins=edges)
    pr = np.diff(stats.norm.cdf(edges / math.sqrt(kT / kappa)))
    pr = pr / pr.sum() * h.sum()
    assert np.sum((h - pr) ** 2 / pr) < 40.0


def test_slot_counts_have_the_stratified_mean():
    """A sweep has floor(x) or floor(x) + 1 slots per layer, x = N (1 - P_F) p_l with p_l the mass
    of the band under Eq. 32, and floor(N P_F) or one more plane waves; the mean over sweeps is x."""
    N, L = 1000, 64.0
    s = I.make_system([], N, L, seed=2)
    o = O.Oracle(params(n_beads=N, box_L=L, lambda_max=32.0, planewave_mode=1, lcut=8, grid_f=8), s.pos, s.chain_len)
    _, _, _, PF = o.pw_modes()
    lo, hi, _, _ = o.layers()
    Nl = 3 / (2.0 ** -3 - 32.0 ** -3)
    x = np.array([N * (1 - PF) * integrate.quad(lambda t: Nl * t ** -4, a, b)[0] for a, b in zip(lo, hi)])
    S = 20000
    c = np.array([o.slot_counts(sw)[0] for sw in range(S)])
    f = np.array([o.slot_counts(sw)[1] for sw in range(S)])
    fl = np.floor(x)
    assert np.all((c == fl) | (c == fl + 1))
    fr = x - fl
    sd = np.sqrt(fr * (1 - fr) / S) + 1e-12
    assert np.all(np.abs(c.mean(0) - x) < 4.5 * sd)
    xf = N * PF
    assert np.all((f == math.floor(xf)) | (f == math.floor(xf) + 1))
    frf = xf - math.floor(xf)
    assert abs(f.mean() - xf) < 4.5 * math.sqrt(frf * (1 - frf) / S)


# ---- full periodic k sampling and the infinite system (Sec. VI.B-C; Appendix D) ----------

def test_k_distribution_cdf_and_its_inverse():
    """P_k^inf (Eq. 52) with N_k^inf = 3 lambda_max^3 / M6 (Eq. 53), in Q = k lambda_max: its CDF
    F(Q) = (3/M6) Int_0^Q q^2 G(q) dq. Checked by swapping the order of integration (scipy):
    Int_0^Q q^2 G = (1/3) Int_0^Q p^6 phi~^2 dp + (Q^3/3) G(Q), with G from scipy; by its
    derivative 3 Q^2 G(Q) / M6; F(inf) = 1. The tabulated inverse maps F(Q) back to Q."""
    M6 = (2 * math.pi) ** 3 / 5
    for Q in (0.7, 2.0, 6.0, 25.0):
        if Q < 2.0:
            inner = integrate.quad(lambda p: p ** 6 * phitilde_by_quadrature(p) ** 2, 0, Q, epsabs=1e-13)[0]
        else:
            inner = (integrate.quad(lambda p: p ** 6 * phitilde_by_quadrature(p) ** 2, 0, 1.0, epsabs=1e-13)[0] +
                     integrate.quad(lambda p: p ** 6 * phitilde_np(p) ** 2, 1.0, Q, limit=400, epsabs=1e-13)[0])
        f = lambda x: x ** 3 * phitilde_np(x) ** 2
        edges = np.arange(Q, 2000.0, math.pi / 2)
        GQ = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-12)[0] for a, b in zip(edges[:-1], edges[1:]))
        GQ += 2 * math.pi ** 2 * edges[-1] ** -4
        want = (inner / 3 + Q ** 3 * GQ / 3) / (M6 / 3)
        assert O.k_cdf_exact(Q) == pytest.approx(want, rel=2e-7)
        h = 1e-4
        dF = (O.k_cdf_exact(Q + h) - O.k_cdf_exact(Q - h)) / (2 * h)
        assert dF == pytest.approx(3 * Q ** 2 * O.G([Q])[0] / M6, rel=1e-5)
    assert O.k_cdf_exact(1e4) == pytest.approx(1.0, abs=2e-4)
    o = O.Oracle(params(n_beads=1, planewave_mode=3), np.array([[1.0, 1, 1]]), np.array([1], np.int32))
    for Q in (0.05, 0.9, 3.3, 47.0, 180.0, 900.0):
        assert o.k_inverse(O.k_cdf_exact(Q)) == pytest.approx(Q, rel=2e-4 if Q < 200 else 2e-2)
    u = np.linspace(1e-6, 1 - 1e-6, 2001)
    q = np.array([o.k_inverse(x) for x in u])
    assert np.all(np.diff(q) > 0)


def test_solid_angle_of_a_sphere_inside_a_cube():
    """The corner correction of the shell: for c < u <= c sqrt 2 the sphere of radius u loses six
    non-overlapping caps, leaving 4 pi (3 c/u - 2); at u >= c sqrt 3 nothing is left; brute
    force by sampling directions otherwise."""
    for t in (1.0, 0.95, 0.8, 0.72):
        assert O.solid_angle_in_cube(t) == pytest.approx(4 * math.pi * (3 * t - 2), rel=1e-6, abs=1e-9)
    assert O.solid_angle_in_cube(1 / math.sqrt(3)) == pytest.approx(0.0, abs=1e-12)
    n = np.random.default_rng(2).normal(size=(2_000_000, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    for t in (0.68, 0.63, 0.6):
        frac = np.mean(np.all(np.abs(n) <= t, axis=1))
        assert O.solid_angle_in_cube(t) / (4 * math.pi) == pytest.approx(frac, abs=4 * math.sqrt(frac / len(n)) + 1e-5)


def test_full_periodic_normalisation_is_the_lattice_sum():
    """Appendix D's discrete cube (|l_i| <= N_layers) plus quasi-continuous shell: the shell's
    weight (the integral of G over mode space outside the cube) matches the lattice sum of
    G(k_l lambda_max) over the modes outside the cube, and the whole normalisation gives R = 1
    (the lattice sum of G equals its integral when lambda_max <= L/2: the inverse transform of
    G vanishes beyond 2 lambda_max, where the wavelet tensor is the harmonic Oseen tensor), so
    P_F (Eq. 56) reaches the infinite-system value (lambda_min/lambda_max)^3 of Eq. 54 whatever
    N_layers is."""
    for L, lmax, Nl in ((40.0, 20.0, 8), (64.0, 16.0, 6)):
        o = O.Oracle(params(n_beads=1, box_L=L, lambda_max=lmax, planewave_mode=2, lcut=Nl, grid_f=8),
                     np.array([[1.0, 1, 1]]), np.array([1], np.int32))
        modes, prob, R, PF = o.pw_modes()
        p_disc, zc, zs, _ = o.pw_tables()
        assert len(modes) == (2 * Nl + 1) ** 3 and np.abs(modes).max() == Nl
        # lattice sum over a large cube of modes, minus the discrete cube; the far tail in closed form
        M = 60
        r = np.arange(-M, M + 1)
        lx, ly, lz = np.meshgrid(r, r, r, indexing="ij")
        l = np.sqrt(lx ** 2 + ly ** 2 + lz ** 2).ravel()
        outside = (np.maximum(np.maximum(np.abs(lx), np.abs(ly)), np.abs(lz)) > Nl).ravel()
        scale = 2 * math.pi * lmax / L
        ls, inv = np.unique(l[outside], return_inverse=True)
        g = O.G(scale * ls)[inv]
        # beyond the big cube G ~ 2 pi^2 Q^-4: the integral of |u|^-4 outside a cube of half-side a is
        # K / a, K = 6 Int Int_[-1,1]^2 (1 + s^2 + t^2)^-2 ds dt (one face at a time, scaled)
        K = 6 * integrate.dblquad(lambda t_, s_: (1 + s_ * s_ + t_ * t_) ** -2, -1, 1, -1, 1)[0]
        lattice = g.sum() + 2 * math.pi ** 2 / scale ** 4 * K / (M + 0.5)
        assert zs == pytest.approx(lattice, rel=6e-3)     # the continuum stands in for the lattice outside
        assert zc == pytest.approx(O.G(scale * np.sqrt((modes.astype(float) ** 2).sum(1))).sum(), rel=1e-12)
        assert p_disc == pytest.approx(zc / (zc + zs), rel=1e-14)
        assert prob.sum() == pytest.approx(p_disc, rel=1e-12)
        assert R == pytest.approx(1.0, abs=5e-4)
        assert PF == pytest.approx((2.0 / lmax) ** 3, rel=6e-4)
    Rs = []
    for Nl in (4, 8, 15):
        o = O.Oracle(params(n_beads=1, box_L=40.0, lambda_max=20.0, planewave_mode=2, lcut=Nl, grid_f=8),
                     np.array([[1.0, 1, 1]]), np.array([1], np.int32))
        Rs.append(o.pw_modes()[2])
    assert abs(Rs[2] - 1) < abs(Rs[1] - 1) < abs(Rs[0] - 1) < 1e-3


def test_full_periodic_samples_and_mobility():
    """Sampled wave vectors: modes of the cube with their probabilities, shell modes never inside
    the cube and with the shell's radial law; from the sampled modes the periodic self-mobility
    at the default N_layers = 15 is the infinite one times 1 - 2.837 a / L (Eq. 60)."""
    L, A0, lmin, N = 40.0, 0.5, 2.0, 1
    o = O.Oracle(params(n_beads=N, box_L=L, lambda_max=L / 2, planewave_mode=2, lcut=15, grid_f=8),
                 np.array([[1.0, 1, 1]]), np.array([1], np.int32))
    modes, prob, R, PF = o.pw_modes()
    p_disc, zc, zs, _ = o.pw_tables()
    k = np.concatenate([o.sample_pw_k(ctr, 200_000) for ctr in range(5)])
    assert np.all(k == np.round(k))
    inside = np.all(np.abs(k) <= 15, axis=1)
    assert abs(inside.mean() - p_disc) < 4.5 * math.sqrt(p_disc * (1 - p_disc) / len(k))
    # the cube: the frequencies of |l|^2 classes against their summed probabilities
    l2 = (k[inside] ** 2).sum(1).astype(int)
    m2 = (modes.astype(int) ** 2).sum(1)
    cls = np.unique(m2)
    want = np.array([prob[m2 == c].sum() for c in cls]) / p_disc * inside.sum()
    got = np.array([(l2 == c).sum() for c in cls])
    keep = want > 20
    chi2 = np.sum((got[keep] - want[keep]) ** 2 / want[keep])
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4
    # Eq. 60 from the sampled modes: <dr^2>_F = <A_F^2 / 2>, A_F = 2 A0 / (k sqrt(5 N))
    kk = (2 * math.pi / L) ** 2 * (k ** 2).sum(1)
    af2 = np.where(kk > 0, 4 * A0 ** 2 / (5 * N * np.where(kk > 0, kk, 1.0)), 0.0) / 2
    drF, se = af2.mean(), af2.std() / math.sqrt(len(af2))
    Nl_ = 3 / (lmin ** -3 - (L / 2) ** -3)
    drw = 2 / 105 * A0 ** 2 * Nl_ * (1 / lmin - 2 / L)
    total = 6 * A0 ** 2 * lmin ** 2 / 105
    ratio = ((1 - PF) * drw + PF * drF) / total
    a = lmin / O.lambda_a()
    assert ratio == pytest.approx(1 - 2.837 * a / L, abs=4.5 * PF * se / total + 2e-4)


def test_infinite_system_k_law_and_time_step():
    """Infinite system (Sec. VI.B): |k| from P_k^inf through the tabulated inverse, k^ isotropic,
    P_F^inf = (lambda_min/lambda_max)^3 (Eq. 54), and the time identity behind Eq. 57:
    (1 - P_F)<dr^2>_w + P_F <dr^2>_F = 6 A0^2 lambda_min^2 / (105 N), with <dr^2>_F the mean of
    A_F^2 / 2 over the sampled law (Eq. 54 gives 6 A0^2 lambda_max^2 / (105 N))."""
    L, lmax, lmin, A0, N = 64.0, 32.0, 2.0, 0.5, 3
    s = I.make_system([], N, L, seed=4)
    o = O.Oracle(params(n_beads=N, box_L=L, lambda_max=lmax, planewave_mode=3, grid_f=8), s.pos, s.chain_len)
    _, _, R, PF = o.pw_modes()
    assert PF == pytest.approx((lmin / lmax) ** 3, rel=1e-15)
    k = np.concatenate([o.sample_pw_k(ctr, 100_000) for ctr in range(3)]) * (2 * math.pi / L)
    kn = np.linalg.norm(k, axis=1)
    Q = kn * lmax
    qs = np.concatenate([np.linspace(0.05, 30, 600), np.geomspace(30, 5000, 200)])
    Fq = np.array([O.k_cdf_exact(x) for x in qs])
    ecdf = np.searchsorted(np.sort(Q), qs) / len(Q)
    assert np.max(np.abs(ecdf - Fq)) < 1.63 / math.sqrt(len(Q)) * 1.5 + 1e-4
    kh = k / kn[:, None]
    assert np.allclose(kh.T @ kh / len(kh), np.eye(3) / 3, atol=0.006)
    # <A_F^2 / 2> with A_F = 2 A0 / (k sqrt(5 N)), over the law as drawn: u = v^3 on a fine midpoint
    # grid of v through the oracle's inverse table (the random mean has infinite variance; in v the
    # integrand 3 v^2 / Q(v^3)^2 is smooth at 0)
    v = (np.arange(400_000) + 0.5) / 400_000
    qq = np.array([o.k_inverse(x) for x in v ** 3])
    drF = np.mean(3 * v ** 2 * 4 * A0 ** 2 / (5 * N * (qq / lmax) ** 2)) / 2
    assert drF == pytest.approx(6 * A0 ** 2 * lmax ** 2 / (105 * N), rel=3e-3)
    Nl_ = 3 / (lmin ** -3 - lmax ** -3)
    drw = 2 / 105 * A0 ** 2 * Nl_ * (1 / lmin - 1 / lmax) / N
    assert (1 - PF) * drw + PF * drF == pytest.approx(6 * A0 ** 2 * lmin ** 2 / (105 * N), rel=3e-3)
    assert o.stats().dt_move * (lmin / O.lambda_a()) ** 2 == pytest.approx(6 * A0 ** 2 * lmin ** 2 / (105 * N), rel=1e-12)


def test_acceptance_laws_metropolis_and_glauber():
    """The acceptance test on each move's draw: accept iff dU <= threshold. For a fixed dU the
    acceptance probability is P(threshold >= dU): min(1, exp(-dU/kT)) for Metropolis (Eq. 20)
    and 1 / (1 + exp(dU/kT)) for Glauber (the alternative of Secs. V.C and VIII)."""
    kT = 1.7
    for acc, law in ((0, lambda x: np.minimum(1.0, np.exp(-x / kT))), (1, lambda x: 1 / (1 + np.exp(x / kT)))):
        o = O.Oracle(params(n_beads=1, kT=kT, acceptance=acc), np.array([[1.0, 1, 1]]), np.array([1], np.int32))
        thr = np.concatenate([o.sample_threshold(sw, 50_000) for sw in range(4)])
        assert np.all(np.isfinite(thr))
        # the survival function of the threshold is the acceptance probability
        assert stats.kstest(-thr, lambda y: law(-np.asarray(y))).pvalue > 1e-3
        for x in (-2.0, 0.0, 0.5, 3.0):
            p_acc = np.mean(thr >= x)
            assert abs(p_acc - law(x)) < 4.5 * math.sqrt(law(x) * (1 - law(x)) / len(thr)) + 1e-12
    assert np.mean(thr >= 0.0) == pytest.approx(0.5, abs=0.005)   # Glauber: a null move half the time


def test_uniform_centres_are_uniform_and_empty_balls_still_count():
    """Uniform centring: moves happen whether or not a bead is inside the ball (time advances
    with each accepted move, Eq. 34); in a dilute box most small balls are empty."""
    N, L = 8, 64.0
    s = I.make_system([], N, L, seed=3)
    o = O.Oracle(params(n_beads=N, box_L=L, seed=5, centring=1), s.pos, s.chain_len)
    o.sweep(200)
    st = o.stats()
    out, n = o.trace_layer(0)
    assert np.mean(n == 0) > 0.9
    assert st.accepted_total == sum(st.attempts)          # free beads: every move accepted (Metropolis)


# ---- wavelet parameter recycling (Appendix D) ----------------------------------------------

def _accepted_and_attempted_lambda(n_chains, grid0, sweeps):
    """lambda of every accepted and every attempted layer-0 wavelet move of dense chains
    (volume fraction 0.15, A0 = 1: acceptance about 0.2, falling across the band)."""
    s = I.make_system([16] * n_chains, 0, I.box_for_volume_fraction(16 * n_chains, 0.15), seed=4)
    L = s.box_L
    p = params(n_beads=s.n_beads, box_L=L, lambda_max=L / 2, A0=1.0, bond_type=1, bond_k=100.0, wca_eps=1.0,
               grid_f=int(L / 2.3), seed=9, grid_layer=[grid0] + [0] * 15)
    o = O.Oracle(p, s.pos, s.chain_len)
    acc, att, deferred = [], [], 0
    for _ in range(sweeps):
        o.sweep(1)
        out, _ = o.trace_layer(0)
        lam = o.trace_lam(0)
        done = (out & 3) != 0
        acc.append(lam[(out & 3) == 1])
        att.append(lam[done])
        deferred += int(((out & 4) != 0).sum())
    o.close()
    att = np.concatenate(att)
    return np.concatenate(acc), att, deferred / len(att), p["lambda_min"]


@pytest.mark.parametrize("n_chains,grid0,sweeps", [(64, 0, 40), (192, 2, 10)])
def test_wavelet_lambda_recycling_keeps_the_accepted_law(n_chains, grid0, sweeps):
    """Appendix D, parameter recycling: a rejected wavelet's lambda is used again by the next
    attempt until it is accepted, so every drawn lambda ends in exactly one accepted move and the
    accepted lambdas follow the drawn law (Eq. 32 on the layer's band) however strongly the
    acceptance depends on lambda; the attempts lean towards the lambdas that are rejected more.
    Serial schedule, and a coloured layer 0 whose carries stay in their queues across sweeps
    (with deferrals rare: a deferred slot runs its own lambda or the serial carry)."""
    acc, att, deferred, lo = _accepted_and_attempted_lambda(n_chains, grid0, sweeps)
    hi = 2 * lo
    F = lambda x: (lo ** -3 - x ** -3) / (lo ** -3 - hi ** -3)
    assert len(acc) > 4000 and np.all((att >= lo) & (att < hi))
    # the acceptance per attempt falls across the band by more than half: without recycling the
    # accepted lambdas would lean to the low end by that much
    q_att = np.floor(F(att) * 4).astype(int)
    q_acc = np.floor(F(acc) * 4).astype(int)
    pacc = [(q_acc == k).sum() / (q_att == k).sum() for k in range(4)]
    assert pacc[0] > 1.8 * pacc[3]
    assert stats.kstest(acc, F).pvalue > 1e-3
    assert stats.kstest(att, F).pvalue < 1e-9
    assert deferred < 0.01
