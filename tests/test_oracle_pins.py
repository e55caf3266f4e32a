"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics,
not by the oracle itself.  CPU only.

Each test names the step it pins and the plausible mistake it catches.
"""

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from helpers import binned_mean_err, circ_dist, load_kat

SEED = 0x5EED2012


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    """Philox4x32-10 against its published known-answer vectors (Salmon et
    al., SC'11): catches a wrong multiplier, Weyl constant, word order or
    round count."""
    for ctr, key, want in load_kat():
        got = oracle.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


def test_philox_uniformity_and_serial_correlation():
    """The 24-bit uniforms of the Metropolis stream are uniform (chi^2 over
    64 bins) and serially uncorrelated (lag-1 correlation of the proposal
    and accept words)."""
    w = oracle.draw_words((32, 32, 16), SEED, 3, 0, oracle.TAG_MET, 7)
    u = (w >> 8).astype(np.float64) / 2.0 ** 24
    assert u.min() >= 0.0 and u.max() < 1.0
    for col in range(2):
        h, _ = np.histogram(u[:, col], bins=64, range=(0.0, 1.0))
        chi2 = ((h - len(u) / 64) ** 2 / (len(u) / 64)).sum()
        assert stats.chi2.sf(chi2, 63) > 1e-4
    r = np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]
    assert abs(r) < 5.0 / np.sqrt(len(u))
    r01 = np.corrcoef(u[:, 0], u[:, 1])[0, 1]
    assert abs(r01) < 5.0 / np.sqrt(len(u))


def test_stream_layout_pairs_sites():
    """Counter layout: packed sites 2q and 2q+1 of one colour share the call
    with ctr0 = q; the even one takes words (0,1), the odd one (2,3); ctr3
    carries slot << 4 | colour << 3 | tag."""
    Lx, Ly, Lz = 8, 4, 2
    seed, slot, colour, count = 0x0123456789ABCDEF, 5, 1, (1 << 40) + 3
    w = oracle.draw_words((Lx, Ly, Lz), seed, slot, colour, oracle.TAG_MET, count)
    n = 0
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                if (x + y + z) % 2 != colour:
                    continue
                p = (x >> 1) + (Lx // 2) * (y + Ly * z)
                ctr = [p >> 1, count & 0xFFFFFFFF, count >> 32,
                       (slot << 4) | (colour << 3) | oracle.TAG_MET]
                key = [seed & 0xFFFFFFFF, seed >> 32]
                ref = oracle.philox4x32_10(ctr, key)
                want = ref[2:4] if p & 1 else ref[0:2]
                assert list(w[n]) == list(want)
                n += 1


# ---------------------------------------------------------------- initial state

_M0, _M1 = 0xD2511F53, 0xCD9E8D57      # Philox4x32 multipliers (SC'11, Table 2)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85      # Weyl key increments (SC'11, Sec. 3.3)


def _philox_py(ctr, key):
    """Philox4x32-10 in plain Python integers, written from the SC'11
    definition independently of the oracle's C: ten rounds of
    (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
    lo(M0 c0)), the key advanced by the Weyl increments between rounds."""
    c0, c1, c2, c3 = (int(v) for v in ctr)
    k0, k1 = (int(v) for v in key)
    m = 0xFFFFFFFF
    for _ in range(10):
        p0, p1 = _M0 * c0, _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & m, p1 & m, ((p0 >> 32) ^ c3 ^ k1) & m, p0 & m
        k0, k1 = (k0 + _W0) & m, (k1 + _W1) & m
    return c0, c1, c2, c3


def test_init_matches_the_stream_definition():
    """The initial state (the hot start of every workload) is theta = 2 pi u
    with u = (w >> 8) 2^-24 from the proposal word of the INIT stream at
    count 0: word 0 of the call with ctr0 = p >> 1 for an even packed index
    p, word 2 for an odd one; ctr3 = slot << 4 | colour << 3 | TAG_INIT.
    Expected angles come from a plain-Python Philox (itself checked on the
    published known answers first), not from the oracle: catches theta =
    pi u, the acceptance word taken for the proposal, a wrong tag, colour or
    slot in the counter, or a swapped pairing."""
    for ctr, key, want in load_kat():
        assert list(_philox_py(ctr, key)) == want
    Lx, Ly, Lz = 6, 4, 4
    for seed, slot in ((SEED, 0), (0x0123456789ABCDEF, 5)):
        th = oracle.init_uniform((Lx, Ly, Lz), seed, slot)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    colour = (x + y + z) % 2
                    p = (x >> 1) + (Lx // 2) * (y + Ly * z)
                    w = _philox_py((p >> 1, 0, 0, (slot << 4) | (colour << 3) | oracle.TAG_INIT), key)
                    u = (w[2 if p & 1 else 0] >> 8) / 2.0 ** 24
                    assert th[z, y, x] == 2 * np.pi * u, (x, y, z)


def test_init_is_uniform_and_uncorrelated():
    """What a hot start must be, whatever the stream: i.i.d. uniform angles
    on [0, 2 pi).  Checked per colour and slot: chi^2 over 64 bins of
    [0, 2 pi) (catches a half or doubled range), <cos theta> = <sin theta> =
    0 within 4 sigma = 4/sqrt(2n), the lattice energy within 4 sigma of its
    beta = 0 law (mean 0, variance 3N/2: the 3N bond cosines of independent
    uniform angles are uncorrelated, each of variance 1/2; catches
    neighbouring sites drawing the same or correlated words) and distinct
    slots uncorrelated."""
    L = 32
    N = L ** 3
    ths = [oracle.init_uniform((L, L, L), SEED, slot) for slot in range(3)]
    z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
    for th in ths:
        assert th.min() >= 0.0 and th.max() < 2 * np.pi
        for colour in (0, 1):
            t = th[((x + y + z) % 2) == colour]
            n = t.size
            h, _ = np.histogram(t, bins=64, range=(0.0, 2 * np.pi))
            chi2 = ((h - n / 64) ** 2 / (n / 64)).sum()
            assert stats.chi2.sf(chi2, 63) > 1e-4
            assert abs(np.cos(t).mean()) < 4 / np.sqrt(2 * n)
            assert abs(np.sin(t).mean()) < 4 / np.sqrt(2 * n)
        assert abs(oracle.measure(th).E) < 4 * np.sqrt(1.5 * N)
    for a, b in ((0, 1), (1, 2)):
        r = np.mean(np.cos(ths[a] - ths[b]))
        assert abs(r) < 4 / np.sqrt(2 * N)


# ---------------------------------------------------------------- measurement

def test_measure_plane_wave_closed_form():
    """Eqs. (4)-(6) sums on a plane wave theta = 2 pi n.r / L, where every
    bond along mu has theta_i - theta_{i+mu} = -2 pi n_mu / L_mu:
    C_mu = N cos(2 pi n_mu / L_mu), S_mu = -N sin(2 pi n_mu / L_mu), M = 0.
    Distinct n_mu and L_mu catch an axis mix-up or a wrong bond sign."""
    Lx, Ly, Lz = 8, 6, 4
    n = (1, 2, 1)
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    th = np.mod(2 * np.pi * (n[0] * x / Lx + n[1] * y / Ly + n[2] * z / Lz), 2 * np.pi)
    th = np.ascontiguousarray(th)
    s = oracle.measure(th)
    N = Lx * Ly * Lz
    for mu, Lm in enumerate((Lx, Ly, Lz)):
        assert s.C[mu] == pytest.approx(N * np.cos(2 * np.pi * n[mu] / Lm), abs=1e-9)
        assert s.S[mu] == pytest.approx(-N * np.sin(2 * np.pi * n[mu] / Lm), abs=1e-9)
    assert abs(s.Mx) < 1e-9 and abs(s.My) < 1e-9
    assert s.E == pytest.approx(-s.C.sum(), abs=1e-12)


def test_measure_ordered_state_and_ring():
    """theta = a everywhere: E = -3N (3 bonds per site), M = N (cos a, sin a);
    on an L x 1 x 1 ring only the x bonds exist (E = -L)."""
    a = 0.7
    th = np.full((4, 6, 8), a)
    s = oracle.measure(th)
    N = th.size
    assert s.E == pytest.approx(-3 * N)
    assert s.Mx == pytest.approx(N * np.cos(a)) and s.My == pytest.approx(N * np.sin(a))
    ring = np.full((1, 1, 10), a)
    r = oracle.measure(ring)
    assert r.E == pytest.approx(-10) and r.C[1] == 0 and r.C[2] == 0


# ---------------------------------------------------------------- over-relaxation

def _local_energy(th):
    """-S_i . sum_j S_j per site, neighbours by periodic rolls (3D)."""
    c, s = np.cos(th), np.sin(th)
    hx = sum(np.roll(c, sh, ax) for ax in range(3) for sh in (1, -1))
    hy = sum(np.roll(s, sh, ax) for ax in range(3) for sh in (1, -1))
    return -(c * hx + s * hy)


def test_overrelax_conserves_energy_and_is_an_involution():
    """Eq. (2): the reflection keeps every updated site's local energy
    (Sec. II: 'exactly the same energy'), moves almost every spin (so it is
    not the identity, the only other energy-keeping map of a unit vector
    with the same field projection), and applied twice with the field frozen
    returns the start."""
    th0 = oracle.init_uniform((8, 8, 8), SEED, 0)
    z, y, x = np.meshgrid(*(np.arange(8),) * 3, indexing="ij")
    for colour in (0, 1):
        mask = ((x + y + z) % 2) == colour
        th = th0.copy()
        e0 = _local_energy(th)
        E0 = oracle.measure(th).E
        oracle.overrelax_half(th, colour)
        e1 = _local_energy(th)
        assert np.max(np.abs(e1 - e0)[mask]) < 1e-12
        assert oracle.measure(th).E == pytest.approx(E0, rel=1e-13)
        moved = circ_dist(th, th0)[mask]
        assert np.mean(moved > 1e-6) > 0.99
        assert np.all(circ_dist(th, th0)[~mask] == 0)
        oracle.overrelax_half(th, colour)
        assert np.max(circ_dist(th, th0)) < 1e-12
        assert th.min() >= 0.0 and th.max() < 2 * np.pi


# ---------------------------------------------------------------- Metropolis

def test_metropolis_single_spin_von_mises():
    """A spin in a fixed field h (its six neighbours frozen at angle a) under
    repeated Metropolis updates samples p(theta) ~ exp(beta |h| cos(theta - a))
    (the von Mises law, kappa = 6 beta): <cos(theta - a)> = I1/I0 and a chi^2
    histogram test.  Catches a wrong dE sign, a missing beta, a proposal not
    uniform, or an accept rule that is not Metropolis."""
    a, beta = 1.0, 0.3
    kappa = 6 * beta
    L = 8
    th = np.full((L, L, L), a)
    z, y, x = np.meshgrid(*(np.arange(L),) * 3, indexing="ij")
    mask = ((x + y + z) % 2) == 0
    samples = []
    for mp in range(2500):
        oracle.metropolis_half(th, beta, SEED, 0, mp, 0)
        if mp >= 100:
            samples.append(th[mask].copy())
    smp = np.array(samples)                        # (passes, sites)
    d = np.mod(smp - a + np.pi, 2 * np.pi) - np.pi
    m, err = binned_mean_err(np.cos(d).mean(axis=1), n_bins=40)
    want = special.i1(kappa) / special.i0(kappa)
    assert abs(m - want) < 5 * err + 1e-4, (m, want, err)
    thin = d[::10].ravel()
    edges = np.linspace(-np.pi, np.pi, 37)
    obs, _ = np.histogram(thin, bins=edges)
    cdf = stats.vonmises.cdf(edges, kappa)
    exp = np.diff(cdf) * len(thin)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2, 35) > 1e-4, chi2


def test_metropolis_beta_zero_iid_moments():
    """beta = 0: every proposal is accepted (u < exp(0) = 1), so each sweep
    leaves i.i.d. uniform spins: <E> = 0, <|M|^2> = N, <|M|^4> = 2N^2 - N,
    U_L = 1/3 + 1/(3N)."""
    L = 8
    N = L ** 3
    th = oracle.init_uniform((L, L, L), SEED, 1)
    acc, ser = oracle.run_chain(th, 0.0, SEED, 1, 0, 1, 0, 4000, 1)
    assert acc == 4000 * N
    M2 = ser[:, 1] ** 2 + ser[:, 2] ** 2
    m, e = binned_mean_err(M2 / N)
    assert abs(m - 1.0) < 4 * e
    m4, e4 = binned_mean_err(M2 ** 2 / (2 * N * N - N))
    assert abs(m4 - 1.0) < 4 * e4
    mE, eE = binned_mean_err(ser[:, 0])
    assert abs(mE) < 4 * eE
    U = 1 - np.mean(M2 ** 2) / (3 * np.mean(M2) ** 2)
    assert abs(U - (1 / 3 + 1 / (3 * N))) < 0.05


def test_high_temperature_energy():
    """beta -> 0: each bond has <cos> = beta/2 + O(beta^3), three bonds per
    site, so <E>/N = -3 beta / 2 + O(beta^3).  Catches a wrong bond count or
    a beta mis-scaling."""
    L, beta = 8, 0.05
    th = oracle.init_uniform((L, L, L), SEED, 2)
    oracle.run_chain(th, beta, SEED, 2, 0, 1, 1, 200, 0)
    _, ser = oracle.run_chain(th, beta, SEED, 2, 200, 1, 1, 6000, 1)
    m, e = binned_mean_err(ser[:, 0] / L ** 3)
    assert abs(m - (-1.5 * beta)) < 4 * e + 3 * beta ** 3, (m, e)
    assert e < 0.1 * 1.5 * beta


@pytest.mark.parametrize("T", [0.01, 0.02, 0.04])
def test_low_temperature_equipartition(T):
    """T -> 0 from the ordered state: one quadratic mode per site (less the
    uniform rotation) gives <E>/N = -3 + (T/2)(1 - 1/N); the quartic term of
    cos adds +T^2/24 (first-order perturbation, <phi_b^2> = T/3 per bond)."""
    L = 8
    N = L ** 3
    beta = 1.0 / T
    th = np.zeros((L, L, L))
    oracle.run_chain(th, beta, SEED, 3, 0, 1, 1, 1500, 0)
    _, ser = oracle.run_chain(th, beta, SEED, 3, 1500, 1, 1, 6000, 1)
    m, e = binned_mean_err(ser[:, 0] / N + 3.0, n_bins=30)
    want = 0.5 * T * (1 - 1 / N) + T * T / 24
    assert abs(m - want) < 4 * e + 0.01 * want, (T, m, want, e)


# ---------------------------------------------------------------- whole chain: ring

def ring_exact(L, beta, nmax=80):
    """L x 1 x 1 periodic ring: Z = (2 pi)^L sum_n I_n(beta)^L.
    <E> = -L sum_n I_n^{L-1} I_n' / sum_n I_n^L, I_n' = (I_{n-1}+I_{n+1})/2;
    rho_s = (1/N)(<C> - beta <S^2>) = (L / beta) sum_n n^2 I_n^L / sum_n I_n^L
    (second derivative of log Z in a twist spread over the L bonds)."""
    n = np.arange(-nmax, nmax + 1, dtype=np.float64)
    I = special.iv(n, beta)
    Ip = 0.5 * (special.iv(n - 1, beta) + special.iv(n + 1, beta))
    Z = np.sum(I ** L)
    return -L * np.sum(I ** (L - 1) * Ip) / Z, (L / beta) * np.sum(n * n * I ** L) / Z


def test_ring_formula_against_quadrature():
    """The Bessel forms themselves, checked by direct integration over the
    ring's angles at L = 3 and L = 4 (theta_0 = 0 by rotation symmetry;
    trapezoid rule on a periodic analytic integrand)."""
    beta = 0.9
    for L, M in ((3, 256), (4, 48)):
        g = np.linspace(0, 2 * np.pi, M, endpoint=False)
        grids = np.meshgrid(*([g] * (L - 1)), indexing="ij")
        th = [np.zeros_like(grids[0])] + list(grids)
        C = sum(np.cos(th[i] - th[(i + 1) % L]) for i in range(L))
        S = sum(np.sin(th[i] - th[(i + 1) % L]) for i in range(L))
        w = np.exp(beta * C)
        Z = w.sum()
        E = -(w * C).sum() / Z
        rho = ((w * C).sum() / Z - beta * (w * S * S).sum() / Z) / L
        Eb, rb = ring_exact(L, beta)
        assert E == pytest.approx(Eb, rel=1e-10)
        assert rho == pytest.approx(rb, rel=1e-10)
    assert ring_exact(3, 0.9)[0] == pytest.approx(-1.57013, abs=1e-5)
    assert ring_exact(3, 0.9)[1] == pytest.approx(0.41965, abs=1e-5)


@pytest.mark.parametrize("beta", [0.5, 1.2])
def test_ring_chain_matches_bessel(beta):
    """Metropolis + over-relaxation sweeps of an 8 x 1 x 1 ring sample the
    exact ring ensemble: <E> and rho_s within 4 sigma of the Bessel forms."""
    L = 8
    th = oracle.init_uniform((L, 1, 1), SEED, 4)
    oracle.run_chain(th, beta, SEED, 4, 0, 1, 1, 1000, 0)
    _, ser = oracle.run_chain(th, beta, SEED, 4, 1000, 1, 1, 200000, 1)
    Eb, rb = ring_exact(L, beta)
    m, e = binned_mean_err(ser[:, 0], n_bins=100)
    assert abs(m - Eb) < 4 * e, (m, Eb, e)
    C, S = ser[:, 3], ser[:, 6]
    mC, eC = binned_mean_err(C)
    mS2, eS2 = binned_mean_err(S * S)
    rho = (mC - beta * mS2) / L
    erho = np.hypot(eC, beta * eS2) / L
    assert abs(rho - rb) < 4 * erho, (rho, rb, erho)


# ---------------------------------------------------------------- parallel tempering

def test_pt_acceptance_is_eq3():
    """Eq. (3): a pair whose hotter replica holds the higher energy swaps
    with probability exp((beta_k - beta_{k+1})(E_k - E_{k+1})) (binomial
    test); the reverse order always swaps."""
    betas = np.array([0.4, 0.5])
    E = np.array([-90.0, -100.0])
    n, acc = 20000, 0
    for t in range(n):
        perm = np.array([0, 1], dtype=np.int32)
        a, _ = oracle.pt_swap(betas, E, perm, SEED, 0, t, 0)
        acc += a
        assert list(perm) == ([1, 0] if a else [0, 1])
    p = np.exp(-1.0)
    assert abs(acc / n - p) < 4 * np.sqrt(p * (1 - p) / n)
    for t in range(200):
        perm = np.array([0, 1], dtype=np.int32)
        a, _ = oracle.pt_swap(betas, E[::-1].copy(), perm, SEED, 0, t, 0)
        assert a == 1


def test_pt_parity_pairs():
    """Even events try pairs (0,1),(2,3); odd events try (1,2),(3,4)."""
    betas = np.linspace(0.40, 0.48, 5)
    E = -np.arange(5, dtype=np.float64) * -10.0        # colder slots hold higher E: always swap
    perm = np.arange(5, dtype=np.int32)
    n, acc = oracle.pt_swap(betas, E, perm, SEED, 0, 0, 0)
    assert n == 2 and list(perm) == [1, 0, 3, 2, 4] and list(acc) == [1, 0, 1, 0, 0]
    perm = np.arange(5, dtype=np.int32)
    n, acc = oracle.pt_swap(betas, E, perm, SEED, 0, 0, 1)
    assert n == 2 and list(perm) == [0, 2, 1, 4, 3]


def test_pt_ladder_of_rings_samples_each_beta():
    """The full exchange machinery on a ladder of four 6-site rings: the
    records filed under each beta match that beta's exact ring energy.  A
    wrong sign in Eq. (3), a swap of configurations without their labels or
    a stale energy biases the per-beta means."""
    betas = np.array([0.4, 0.7, 1.0, 1.3])
    sim = oracle.Simulation.create([(6, 1, 1)], [4], betas, SEED)
    sim.run(1, 1, 300, 0, 1)
    sim.records.clear()
    sim.run(1, 1, 12000, 1, 1)
    by_k = {k: [] for k in range(4)}
    for r in sim.records:
        by_k[r.beta_index].append(r.sums.E)
    for k, b in enumerate(betas):
        m, e = binned_mean_err(np.array(by_k[k]), n_bins=40)
        assert abs(m - ring_exact(6, b)[0]) < 4 * e, (b, m, e)
    assert all(a.sum() > 100 for a in sim.swap_accepts)


# ---------------------------------------------------------------- reweighting

def _series(T, seed=11, L=8):
    from paper_1211_0780_b300.inputs import synthetic_series
    s = synthetic_series(L, T, seed)
    O = np.stack([s["m2"].astype(np.float64), s["m4"].astype(np.float64),
                  s["c"].astype(np.float64).sum(0), s["s2"].astype(np.float64).sum(0)], axis=1)
    return s, O


def test_reweight_identity_at_beta0():
    """beta' = beta0: the weights are uniform, so the reweighted means are
    the plain means and log Z = log T."""
    s, O = _series(5000)
    logZ, mE, mean, cov = oracle.reweight(s["E"], O, 0.4542, [0.4542])
    assert logZ[0] == pytest.approx(np.log(5000), rel=1e-14)
    assert mE[0] == pytest.approx(s["E"].mean(), rel=1e-13)
    np.testing.assert_allclose(mean[0], O.mean(axis=0), rtol=1e-13)
    c_plain = (O * s["E"][:, None]).mean(0) - O.mean(0) * s["E"].mean()
    np.testing.assert_allclose(cov[0], c_plain, rtol=1e-8)


def test_reweight_brute_force_multiprecision():
    """Against a 40-digit evaluation of the same sums (no max shift), T = 1000."""
    import mpmath as mp
    mp.mp.dps = 40
    s, O = _series(1000)
    bp = [0.4530, 0.4549, 0.4555]
    logZ, mE, mean, cov = oracle.reweight(s["E"], O, 0.4542, bp)
    for k, b in enumerate(bp):
        db = mp.mpf(b) - mp.mpf(0.4542)
        w = [mp.e ** (-db * mp.mpf(float(e))) for e in s["E"]]
        Z = mp.fsum(w)
        assert logZ[k] == pytest.approx(float(mp.log(Z)), rel=1e-13)
        Em = mp.fsum(wi * mp.mpf(float(e)) for wi, e in zip(w, s["E"])) / Z
        assert mE[k] == pytest.approx(float(Em), rel=1e-13)
        for j in range(O.shape[1]):
            Om = mp.fsum(wi * mp.mpf(float(o)) for wi, o in zip(w, O[:, j])) / Z
            OEm = mp.fsum(wi * mp.mpf(float(o)) * mp.mpf(float(e))
                          for wi, o, e in zip(w, O[:, j], s["E"])) / Z
            assert mean[k, j] == pytest.approx(float(Om), rel=1e-12)
            assert cov[k, j] == pytest.approx(float(OEm - Om * Em), rel=1e-7, abs=1e-12)


def test_reweight_derivative_matches_finite_difference():
    """d<O>/dbeta' = -(<O E> - <O><E>) against a central difference, and the
    chain rule to U_L and rho_s L (including rho_s's explicit beta' factor)
    against central differences of those functions."""
    s, O = _series(20000, L=16)
    b = np.array([0.4533, 0.4548])
    h = 1e-6
    _, _, mean, cov = oracle.reweight(s["E"], O, 0.4542, b)
    _, _, mp_, _ = oracle.reweight(s["E"], O, 0.4542, b + h)
    _, _, mm_, _ = oracle.reweight(s["E"], O, 0.4542, b - h)
    fd = (mp_ - mm_) / (2 * h)
    np.testing.assert_allclose(-cov, fd, rtol=1e-6)
    args = (s["E"], s["m2"], s["m4"], s["c"].T, s["s2"].T, 0.4542)
    r0 = oracle.reweight_observables(*args, b, 16)
    rp = oracle.reweight_observables(*args, b + h, 16)
    rm = oracle.reweight_observables(*args, b - h, 16)
    for key, dkey in (("U", "dU"), ("rhoL", "drhoL")):
        np.testing.assert_allclose(r0[dkey], (rp[key] - rm[key]) / (2 * h), rtol=1e-6)


@pytest.mark.parametrize("T", [1, 777])
def test_reweight_constant_energy_closed_forms(T):
    """Constant energy E0: equal weights at every beta', so the averages are
    the plain means, log Z = log T - (beta' - beta0) E0, the covariances
    vanish, dU/dbeta' = 0 and d(rho_s L)/dbeta' = -(L/3) <s2> (Eq. 6's
    explicit beta' alone).  A sign slip in that explicit term, or in the
    shift of log Z, fails here."""
    rng = np.random.default_rng(T)
    L, beta0, E0 = 8, 0.4542, -1234.5
    m2 = rng.random(T)
    c, s2 = rng.random((T, 3)), rng.random((T, 3))
    bp = np.array([0.440, beta0, 0.470])
    r = oracle.reweight_observables(np.full(T, E0), m2, m2 * m2, c, s2, beta0, bp, L)
    m2m, m4m, cm, s2m = m2.mean(), (m2 * m2).mean(), c.sum(1).mean(), s2.sum(1).mean()
    np.testing.assert_allclose(r["logZ"], np.log(T) - (bp - beta0) * E0, rtol=1e-13, atol=1e-10)
    np.testing.assert_allclose(r["E"], E0, rtol=1e-13)  # T additions of w E0: T eps at most
    np.testing.assert_allclose(r["U"], 1.0 - m4m / (3.0 * m2m * m2m), rtol=1e-13)
    np.testing.assert_allclose(r["rhoL"], L / 3.0 * (cm - bp * s2m), rtol=1e-13)
    # the covariances <O E> - <O><E> cancel terms of size |E0| <O> ~ 10^3 to ~1e-12
    np.testing.assert_allclose(r["dU"], 0.0, atol=1e-10)
    np.testing.assert_allclose(r["drhoL"], -L / 3.0 * s2m, rtol=0, atol=1e-10)
