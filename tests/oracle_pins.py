"""Pins of the FP64 oracle: checks against facts fixed by the paper and by mathematics,
not by the oracle's own code.

Each function raises AssertionError when the oracle (whichever build of it is loaded)
disagrees with the fact it pins.  tests/test_oracle_pins.py runs them against the
oracle; tests/test_oracle_mutants.py runs them against copies of the oracle with a
planted mistake and requires that some pin fails for every mistake.

Facts used (paper: arXiv 2412.14775, Sections 2.1, 2.2, Tables 1-2):
  P1  SK under the null.  If |I_i| are i.i.d. Gamma(shape d), the generalised
      spectral kurtosis of Nita & Gary (2010; cited in Sec. 2.1) has E[tau] = 1 and
      Var[tau] = 2 d (d+1) W^2 / ((W-1)(Wd+2)(Wd+3)).  (The Dirichlet moments of
      |I_i|/S1 give both; d = 1 is the classic 4W^2/((W-1)(W+2)(W+3)).)
  P2  Cauchy-Schwarz: 1 <= W S2/S1^2 <= W, so 0 <= tau <= Wd+1, with tau = 0 for a
      constant magnitude and tau = Wd+1 for a single non-zero sample.
  P3  A fully polarised signal V = c e e^H has (Q, U, V) = c w with a fixed real w,
      |w| = |e1|^2 + |e2|^2 = I/c, so both directional statistics are 1.
  P4  Isotropic noise: unit vectors uniform on the sphere, E[r^2] = 1/W exactly;
      antipodal pairs give r = 0.
  P5  Hermitian autocorrelations have Im Q = Im U = Im V = 0, so r_Im = 0.
  P6  Averaging: mean of unflagged samples and weight n/K, checked over every subset
      of flagged windows of a bin.
  P7  Exact evaluation on a small integer grid (50-digit arithmetic, Stokes taken as
      traces against the Pauli matrices instead of the sums of Eq. IQUV).
  P8  Splitting a stream into blocks at multiples of W changes nothing.
  P10 Windows are runs of consecutive samples of a stream (Sec. 2), whatever the
      correlator's block length: with partial windows, blocks of any length give the
      windows, flags and averages of the unsplit stream, each reported once.
  P11 Online thresholds follow their stated rule (oracle/adaptive.py).
  P12 Symmetries of the definitions: sample order within a window, feed swap, sign,
      conjugation and scale leave the statistics unchanged; a factor j swaps the parts.
  P13 Overlapping windows (an extension): each window is a window of the plain method
      on a shifted stream; a spike flags exactly the samples of the windows holding it;
      averages by brute force; any split at multiples of the hop changes nothing.
"""
import itertools
import math
from fractions import Fraction

import mpmath
import numpy as np

import oracle
from oracle import OracleStream

EPS32 = 2.0 ** -23


def _stream(R, M, K, d=1.0, s_low=-1e300, s_high=1e300, gamma=1e300, eps=EPS32):
    return OracleStream(R, M, K, d, s_low, s_high, gamma, eps)


def _run_windows(vis, M, d=1.0, eps=EPS32, **thr):
    """vis [nwin, M, 4] complex -> oracle outputs with one window per row."""
    st = _stream(vis.shape[0], M, M, d=d, eps=eps, **thr)
    return st.process(vis)


def _sk_var(M, d):
    return 2.0 * d * (d + 1.0) * M * M / ((M - 1.0) * (M * d + 2.0) * (M * d + 3.0))


def _check_mean_var(tau, M, d, z=4.0):
    n = tau.size
    var_cf = _sk_var(M, d)
    mean = tau.mean()
    assert abs(mean - 1.0) < z * math.sqrt(var_cf / n), (M, d, mean)
    c = tau - mean
    v = np.mean(c * c)
    m4 = np.mean(c ** 4)
    se_v = math.sqrt(max(m4 - v * v, 0.0) / n)
    assert abs(v - var_cf) < z * se_v, (M, d, v, var_cf)


# ---------------------------------------------------------------------------------
def pin_p1_sk_null_gamma(nwin=100000, seed=1):
    """P1 with |I| ~ Gamma(d): xx carries the positive real magnitude, all else 0."""
    for M, d in ((16, 1.0), (16, 2.0), (20, 0.5), (8, 3.66)):
        rng = np.random.default_rng(seed + M * 7 + int(d * 10))
        g = rng.gamma(shape=d, scale=1.0, size=(nwin, M))
        vis = np.zeros((nwin, M, 4), np.complex128)
        vis[..., 0] = g
        out = _run_windows(vis, M, d=d, eps=0.0)
        _check_mean_var(out["tau"].ravel(), M, d)


def pin_p1_sk_null_autocorrelation(nwin=100000, seed=2):
    """P1 with unaveraged autocorrelations of complex Gaussian voltages x, y:
    I = |x|^2 + |y|^2 is Gamma(2) distributed, so d = 2 centres tau at 1."""
    M = 16
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((nwin, M)) + 1j * rng.standard_normal((nwin, M))) / math.sqrt(2)
    y = (rng.standard_normal((nwin, M)) + 1j * rng.standard_normal((nwin, M))) / math.sqrt(2)
    vis = np.stack([x * x.conj(), x * y.conj(), y * x.conj(), y * y.conj()], axis=-1)
    out = _run_windows(vis, M, d=2.0, eps=0.0)
    _check_mean_var(out["tau"].ravel(), M, 2.0)


def pin_p2_sk_bounds(seed=3):
    """P2: 0 <= tau <= Wd+1 on arbitrary data, and both ends are attained."""
    rng = np.random.default_rng(seed)
    for M, d in ((2, 1.0), (5, 0.7), (16, 3.66), (64, 1.0)):
        lead = (M * d + 1.0) / (M - 1.0)
        n = 4000
        mags = np.concatenate([
            rng.lognormal(0.0, 3.0, size=(n, M)),
            rng.uniform(0, 1, size=(n, M)) * (rng.uniform(size=(n, M)) < 0.2),
            rng.exponential(size=(n, M))])
        keep = mags.sum(axis=1) > 0
        mags = mags[keep]
        ph = rng.uniform(0, 2 * np.pi, size=mags.shape)
        vis = np.zeros(mags.shape + (4,), np.complex128)
        vis[..., 0] = mags * np.exp(1j * ph) * 0.5
        vis[..., 3] = mags * np.exp(1j * ph) * 0.5          # I = xx + yy = mags e^{j ph}
        vis[..., 1] = rng.standard_normal(mags.shape)        # xy, yx do not enter SK
        tau = _run_windows(vis, M, d=d, eps=0.0)["tau"].ravel()
        assert np.all(tau >= -1e-12 * (M * d + 1)), (M, d, tau.min())
        assert np.all(tau <= (M * d + 1) * (1 + 1e-12)), (M, d, tau.max())

        # constant magnitude, random phases -> tau = 0 (I split evenly over xx and yy)
        const = np.zeros((50, M, 4), np.complex128)
        const[..., 0] = 1.5 * np.exp(1j * rng.uniform(0, 2 * np.pi, size=(50, M)))
        const[..., 3] = const[..., 0]
        tau0 = _run_windows(const, M, d=d, eps=0.0)["tau"]
        assert np.all(np.abs(tau0) < 1e-12 * lead * M), (M, d, tau0)

        # one non-zero sample -> tau = Wd + 1
        one = np.zeros((M, M, 4), np.complex128)
        for k in range(M):
            one[k, k, 0] = 2.5 - 1.5j
        tau1 = _run_windows(one, M, d=d, eps=0.0)["tau"]
        assert np.allclose(tau1, M * d + 1.0, rtol=1e-13, atol=0), (M, d, tau1)

        # all-zero window with eps > 0: tau = lead * (0/eps - 1) = -lead, finite
        zero = np.zeros((1, M, 4), np.complex128)
        tz = _run_windows(zero, M, d=d, eps=EPS32)["tau"]
        assert tz[0, 0] == -lead, (M, d, tz)


def _polarised(rng, nwin, M, c_of):
    th = rng.uniform(0, np.pi, size=(nwin, 1))
    ph = np.where(rng.uniform(size=(nwin, 1)) < 0.5, 0.0, rng.uniform(0, 2 * np.pi, size=(nwin, 1)))
    e1 = np.cos(th) * np.ones((1, M))
    e2 = np.sin(th) * np.exp(1j * ph) * np.ones((1, M))
    c = c_of(rng, nwin, M)
    return np.stack([c * e1 * e1.conj(), c * e1 * e2.conj(), c * e2 * e1.conj(), c * e2 * e2.conj()],
                    axis=-1)


def pin_p3_fully_polarised(seed=4):
    """P3: a fully polarised window has r_Re = r_Im = 1; a real c has r_Im = 0;
    and per sample |(Re Q, Re U, Re V)| = |Re I| for real c (Stokes identity)."""
    rng = np.random.default_rng(seed)
    M = 16

    def const_phase(rng, n, M):       # varying amplitude, constant phase per window
        amp = rng.uniform(0.5, 20.0, size=(n, M))
        ph = rng.uniform(0, 2 * np.pi, size=(n, 1))
        return amp * np.exp(1j * ph)

    vis = _polarised(rng, 2000, M, const_phase)
    out = _run_windows(vis, M, eps=0.0)
    assert np.allclose(out["r_re"], 1.0, rtol=0, atol=1e-12), out["r_re"].min()
    assert np.allclose(out["r_im"], 1.0, rtol=0, atol=1e-12), out["r_im"].min()

    def real_c(rng, n, M):
        return rng.uniform(0.5, 20.0, size=(n, M)) * np.where(rng.uniform(size=(n, 1)) < 0.5, -1, 1)

    vis = _polarised(rng, 500, M, real_c)
    # with c real, yx = conj(xy) and xx, yy are real; write them so exactly (the
    # products above round differently in the last bit)
    vis[..., 2] = vis[..., 1].conj()
    vis[..., 0] = vis[..., 0].real
    vis[..., 3] = vis[..., 3].real
    out = _run_windows(vis, M, eps=EPS32)
    assert np.all(out["r_im"] == 0.0)
    assert np.allclose(out["r_re"], 1.0, rtol=0, atol=1e-6)
    # c purely imaginary: Re(Q, U, V) = 0 so r_Re = 0, r_Im = 1; only the Im part
    # can raise the flag (the Re and Im flags are combined with OR, Sec. 2.2)
    vis_i = 1j * vis
    out = _run_windows(vis_i, M, eps=EPS32, s_low=-1e300, s_high=1e300, gamma=0.5)
    assert np.all(out["r_re"] == 0.0)
    assert np.allclose(out["r_im"], 1.0, rtol=0, atol=1e-6)
    assert np.all(out["wflag"] == 1)
    for k in range(50):
        s = oracle.stokes(np.stack([vis[k, 0].real, vis[k, 0].imag], -1).reshape(8))
        assert math.isclose(math.hypot(s[2], s[4], s[6]), abs(s[0]), rel_tol=1e-12), s


def pin_p4_isotropic_null(nwin=100000, seed=5):
    """P4: i.i.d. circular Gaussian correlations give E[r^2] = 1/W per part, and a
    window made of antipodal pairs gives r = 0 exactly."""
    rng = np.random.default_rng(seed)
    for M in (8, 16, 20):
        vis = (rng.standard_normal((nwin, M, 4)) + 1j * rng.standard_normal((nwin, M, 4))) / math.sqrt(2)
        out = _run_windows(vis, M, eps=0.0)
        for key in ("r_re", "r_im"):
            r2 = out[key].ravel() ** 2
            se = r2.std() / math.sqrt(r2.size)
            assert abs(r2.mean() - 1.0 / M) < 4 * se, (M, key, r2.mean(), 1.0 / M)
        half = (rng.standard_normal((200, M // 2, 4)) + 1j * rng.standard_normal((200, M // 2, 4)))
        anti = np.empty((200, M, 4), np.complex128)
        anti[:, 0::2] = half
        anti[:, 1::2] = -half
        o2 = _run_windows(anti, M, eps=EPS32)
        assert np.all(o2["r_re"] == 0.0) and np.all(o2["r_im"] == 0.0)


def pin_p5_autocorrelation_r_im(seed=6):
    """P5: Hermitian V (xx, yy real, yx = conj(xy)) gives r_Im = 0 exactly."""
    rng = np.random.default_rng(seed)
    M = 16
    n = 3000
    xx = rng.exponential(size=(n, M))
    yy = rng.exponential(size=(n, M))
    xy = rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))
    vis = np.stack([xx + 0j, xy, xy.conj(), yy + 0j], axis=-1)
    out = _run_windows(vis, M, eps=EPS32)
    assert np.all(out["r_im"] == 0.0)
    assert np.all(out["r_re"] > 0.0)


def pin_p6_averaging_bruteforce(seed=7):
    """P6: for every subset of flagged windows in a bin, the output equals the mean
    of the unflagged samples (numpy), the weight equals their count / K, and the
    per-sample flag bits equal the window flags expanded over W samples."""
    rng = np.random.default_rng(seed)
    for M, nb in ((4, 8), (16, 4), (3, 5)):
        K = M * nb
        d = 1.0
        lead_max = M * d + 1.0
        subsets = list(itertools.product((0, 1), repeat=nb))
        R = len(subsets)
        vis = np.zeros((R, K, 4), np.complex128)
        for rr, sub in enumerate(subsets):
            for w, fl in enumerate(sub):
                blk = vis[rr, w * M:(w + 1) * M]
                # xy, yx never enter SK; gamma = 2 keeps DS from flagging (r <= 1)
                blk[:, 1] = rng.standard_normal(M) + 1j * rng.standard_normal(M)
                blk[:, 2] = rng.standard_normal(M) + 1j * rng.standard_normal(M)
                if fl:     # spike window: I non-zero at one sample only -> tau = Wd + 1
                    blk[rng.integers(M), 0] = 3.0 + 1.0j
                else:      # flat window: |I| constant -> tau = 0
                    blk[:, 0] = 2.0 * np.exp(1j * rng.uniform(0, 2 * np.pi, size=M))
        st = OracleStream(R, M, K, d, -0.5, lead_max / 2, 2.0, EPS32)
        out = st.process(vis)
        want_flags = np.array(subsets, dtype=np.uint8)
        assert np.array_equal(out["wflag"], want_flags), M
        for rr, sub in enumerate(subsets):
            keep = np.repeat(1 - np.array(sub), M).astype(bool)
            n = keep.sum()
            exp = vis[rr][keep].mean(axis=0) if n else np.zeros(4)
            got = out["avg"][rr, 0].reshape(4, 2)
            assert np.allclose(got[:, 0], exp.real, rtol=1e-13, atol=1e-14), (M, sub)
            assert np.allclose(got[:, 1], exp.imag, rtol=1e-13, atol=1e-14), (M, sub)
            assert out["weight"][rr, 0] == n / K
            bits = np.zeros((K + 31) // 32, np.uint64)
            for t in range(K):
                if not keep[t]:
                    bits[t // 32] |= np.uint64(1) << np.uint64(t % 32)
            assert np.array_equal(out["flagbits"][rr].astype(np.uint64), bits), (M, sub)


def _pauli_stokes(v):
    """Stokes (I, Q, U, V) of one 2x2 correlation matrix as traces tr(V sigma_k) with
    sigma = (identity, Z, X, Y) -- a second route to Eq. IQUV."""
    Vm = [[v[0], v[1]], [v[2], v[3]]]
    sig = {
        "I": [[1, 0], [0, 1]], "Q": [[1, 0], [0, -1]],
        "U": [[0, 1], [1, 0]], "V": [[0, -1j], [1j, 0]]}
    out = []
    for k in "IQUV":
        s = sig[k]
        tr = sum(Vm[a][b] * s[b][a] for a in range(2) for b in range(2))
        out.append(complex(tr))
    return out


def pin_p7_exact_grid(nwin_per_M=3000, seed=8):
    """P7: windows of W in {2,3,4} with every correlation on {-1,0,1}+j{-1,0,1};
    statistics to 1e-12 against 50-digit evaluation, flags identical (ties at a
    threshold, decided exactly, are counted and must also agree)."""
    mpmath.mp.dps = 50
    rng = np.random.default_rng(seed)
    eps = Fraction(1, 2 ** 23)
    epsm = mpmath.mpf(1) / 2 ** 23
    for M, d in ((2, 1.0), (3, 0.5), (4, 2.0)):
        s_low, s_high, gamma = 0.25, 1.75, 0.6
        vals = rng.integers(-1, 2, size=(nwin_per_M, M, 4, 2))
        vis = vals[..., 0] + 1j * vals[..., 1]
        out = _run_windows(vis, M, d=d, eps=float(eps), s_low=s_low, s_high=s_high, gamma=gamma)
        dd = Fraction(d)
        lead = (M * dd + 1) / (M - 1)
        for w in range(nwin_per_M):
            st = [_pauli_stokes(vis[w, i]) for i in range(M)]
            # SK: S2 is an exact rational, S1 a sum of square roots of integers
            S2 = sum(Fraction(int(round(s[0].real)) ** 2 + int(round(s[0].imag)) ** 2) for s in st)
            S1 = mpmath.fsum(mpmath.sqrt(int(round(s[0].real)) ** 2 + int(round(s[0].imag)) ** 2)
                             for s in st)
            tau = mpmath.mpf(lead.numerator) / lead.denominator * (
                M * mpmath.mpf(S2.numerator) / S2.denominator / (S1 * S1 + epsm) - 1)
            rs = []
            for part in (0, 1):
                acc = [mpmath.mpf(0)] * 3
                for s in st:
                    comp = [int(round((s[k].real, s[k].imag)[part])) for k in (1, 2, 3)]
                    p = mpmath.sqrt(sum(c * c for c in comp)) + epsm
                    acc = [acc[k] + comp[k] / p for k in range(3)]
                rs.append(mpmath.sqrt(sum(a * a for a in acc)) / M)
            got = (out["tau"][w, 0], out["r_re"][w, 0], out["r_im"][w, 0])
            for g, e, floor in zip(got, (tau, rs[0], rs[1]), (1.0, M ** -0.5, M ** -0.5)):
                assert abs(g - float(e)) <= 1e-12 * max(abs(float(e)), floor), (M, w, g, e)
            f = (tau < s_low) or (tau > s_high) or (rs[0] > gamma) or (rs[1] > gamma)
            assert bool(out["wflag"][w, 0]) == bool(f), (M, w, got)


def pin_p8_block_split(seed=9):
    """P8: processing a stream as one block or as blocks split at multiples of W
    gives identical statistics, flags, averages and weights."""
    rng = np.random.default_rng(seed)
    R, M, K, T = 7, 4, 24, 240
    vis = rng.standard_normal((R, T, 4)) + 1j * rng.standard_normal((R, T, 4))
    vis[:, 50:60] *= 8.0
    vis[2, 100:130, :] = 5.0 * (1 + 1j)
    thr = (1.0, 0.3, 2.0, 0.7, EPS32)
    whole = OracleStream(R, M, K, *thr).process(vis)
    for cuts in ((8, 120), (4, 28, 96, 100, 236), (24, 48, 72), (12,)):
        st = OracleStream(R, M, K, *thr)
        parts = []
        edges = (0,) + cuts + (T,)
        for a, b in zip(edges[:-1], edges[1:]):
            parts.append(st.process(vis[:, a:b]))
        for key in ("tau", "r_re", "r_im", "wflag"):
            assert np.array_equal(np.concatenate([p[key] for p in parts], axis=1), whole[key]), key
        assert np.array_equal(np.concatenate([p["avg"] for p in parts], axis=1), whole["avg"])
        assert np.array_equal(np.concatenate([p["weight"] for p in parts], axis=1), whole["weight"])


ALL_PINS = [pin_p1_sk_null_gamma, pin_p1_sk_null_autocorrelation, pin_p2_sk_bounds,
            pin_p3_fully_polarised, pin_p4_isotropic_null, pin_p5_autocorrelation_r_im,
            pin_p6_averaging_bruteforce, pin_p7_exact_grid, pin_p8_block_split]


def pin_p9_tf_footprints(seed=10):
    """P9: time-frequency footprints (W = M x F samples over F adjacent channels).

    (a) A footprint's statistics depend only on its W samples: they equal, bit for bit,
        those of a time-only window holding the same samples row after row.
    (b) P1 holds with W = M F: Gamma(d) magnitudes over a 8x2 footprint have E[tau] = 1
        and the closed-form variance for W = 16.
    (c) P4 holds with W = M F: isotropic noise over a 5x4 footprint has E[r^2] = 1/20.
    (d) A window flagged by one channel flags every channel of the footprint, and each
        channel's average leaves it out."""
    rng = np.random.default_rng(seed)
    # (a)
    for M, F in ((10, 2), (5, 4), (3, 2)):
        G, nw = 6, 4
        v = rng.standard_normal((G * F, M * nw, 4)) + 1j * rng.standard_normal((G * F, M * nw, 4))
        v[:, :M] *= 5.0
        a = OracleStream(G * F, M, M, 1.0, 0.2, 2.5, 0.5, EPS32, F=F).process(v)
        # rows of w hold, window by window, the F channels' samples one after another
        w = np.stack([np.concatenate([np.concatenate([v[g * F + k, M * t:M * (t + 1)]
                                                      for k in range(F)]) for t in range(nw)])
                      for g in range(G)])
        b = OracleStream(G, M * F, M * F, 1.0, 0.2, 2.5, 0.5, EPS32).process(w)
        for key in ("tau", "r_re", "r_im", "wflag"):
            assert np.array_equal(a[key], b[key]), (M, F, key)
    # (b)
    M, F, d, n = 8, 2, 1.5, 100000
    g = rng.gamma(shape=d, size=(n * F, M))
    vis = np.zeros((n * F, M, 4), np.complex128)
    vis[..., 0] = g
    out = OracleStream(n * F, M, M, d, -1e300, 1e300, 1e300, 0.0, F=F).process(vis)
    _check_mean_var(out["tau"].ravel(), M * F, d)
    # (c)
    M, F, n = 5, 4, 50000
    vis = (rng.standard_normal((n * F, M, 4)) + 1j * rng.standard_normal((n * F, M, 4))) / math.sqrt(2)
    out = OracleStream(n * F, M, M, 1.0, -1e300, 1e300, 1e300, 0.0, F=F).process(vis)
    for key in ("r_re", "r_im"):
        r2 = out[key].ravel() ** 2
        assert abs(r2.mean() - 1.0 / (M * F)) < 4 * r2.std() / math.sqrt(r2.size), key
    # (d)
    M, F, nb = 4, 2, 4
    K = M * nb
    subsets = list(itertools.product((0, 1), repeat=nb))
    G = len(subsets)
    vis = np.zeros((G * F, K, 4), np.complex128)
    for gi, sub in enumerate(subsets):
        for k in range(F):
            row = vis[gi * F + k]
            row[:, 1] = rng.standard_normal(K) + 1j * rng.standard_normal(K)
            row[:, 0] = 2.0 * np.exp(1j * rng.uniform(0, 2 * np.pi, size=K))   # flat |I|
        for w, fl in enumerate(sub):
            if fl:   # a spike in one channel only: that footprint's |I| is no longer flat
                vis[gi * F + 1, w * M + 1, 0] = 40.0
    # a flat footprint has tau = 0; the spiked one has tau = lead * (W*1628/54**2 - 1) > 4
    st = OracleStream(G * F, M, K, 1.0, -0.5, 2.0, 2.0, EPS32, F=F)
    out = st.process(vis)
    assert np.array_equal(out["wflag"], np.array(subsets, dtype=np.uint8))
    for gi, sub in enumerate(subsets):
        keep = np.repeat(1 - np.array(sub), M).astype(bool)
        for k in range(F):
            row = gi * F + k
            bits = sum(1 << t for t in range(K) if not keep[t])
            assert int(out["flagbits"][row, 0]) == bits, (sub, k)
            exp = vis[row][keep].mean(axis=0) if keep.any() else np.zeros(4)
            got = out["avg"][row, 0].reshape(4, 2)
            assert np.allclose(got[:, 0], exp.real, rtol=1e-13, atol=1e-14)
            assert np.allclose(got[:, 1], exp.imag, rtol=1e-13, atol=1e-14)
            assert out["weight"][row, 0] == keep.sum() / K


ALL_PINS.append(pin_p9_tf_footprints)


def _bits(words, n):
    """The first n flag bits of a row's words, bit t of word t // 32 at t mod 32."""
    w = np.asarray(words, dtype=np.uint64)
    return [(int(w[t >> 5]) >> (t & 31)) & 1 for t in range(n)]


def pin_p10_partial_windows(seed=11):
    """P10: blocks of any length (partial windows carried between blocks) give, per
    completed window, exactly the unsplit stream's statistics, flag bits and averages;
    samples of a window still open at the end are not reported."""
    rng = np.random.default_rng(seed)
    for R, M, K, F, T in ((6, 5, 20, 1, 203), (8, 4, 24, 2, 150), (5, 16, 16, 1, 100)):
        vis = rng.standard_normal((R, T, 4)) + 1j * rng.standard_normal((R, T, 4))
        vis[:, 30:41] *= 6.0
        vis[1, 60:95, :] = 4.0 * (1 - 1j)
        thr = (1.0, 0.3, 2.0, 0.7, EPS32)
        whole_T = (T // M) * M
        whole = OracleStream(R, M, K, *thr, F=F).process(vis[:, :whole_T])
        for cuts in ((1, 2, 3, 50, 51, 130), (7, 77), tuple(range(3, T, 13)), (M + 1,)):
            st = OracleStream(R, M, K, *thr, F=F, partial=True)
            edges = (0,) + tuple(c for c in cuts if c < T) + (T,)
            parts = []
            for a, b in zip(edges[:-1], edges[1:]):
                nwin, f0 = st.windows_for(b - a)
                n_out = st.outputs_for(b - a)
                out = st.process(vis[:, a:b])
                assert out["tau"].shape[1] == nwin and out["avg"].shape[1] == n_out
                assert f0 == (a // M) * M if nwin else True
                parts.append(out)
            for key in ("tau", "r_re", "r_im", "wflag"):
                got = np.concatenate([p[key] for p in parts], axis=1)
                assert np.array_equal(got, whole[key]), (M, cuts, key)
            for key in ("avg", "weight"):
                got = np.concatenate([p[key] for p in parts], axis=1)
                assert np.array_equal(got, whole[key]), (M, cuts, key)
            for r in range(R):
                bits = []
                for p in parts:
                    bits += _bits(p["flagbits"][r], p["tau"].shape[1] * M)
                assert bits == _bits(whole["flagbits"][r], whole_T), (M, cuts, r)
            assert st.pending.shape[1] == T - whole_T


ALL_PINS.append(pin_p10_partial_windows)


def _level_windows(levels, M):
    """Rows of windows whose tau is fixed by construction: xx = yy = s/2 real, xy = yx
    = 0, so I = s and Q = U = V = 0 (r = 0, the DS test never flags).  A window of
    constant s has W S2/S1^2 = 1; one alternating s = 1, 3 has W S2/S1^2 = 5/4."""
    out = []
    for lev in levels:
        s = np.ones(M) if lev == "A" else np.tile([1.0, 3.0], M // 2)
        out.append(s)
    s = np.concatenate(out)
    vis = np.zeros((1, s.size, 4), np.complex128)
    vis[0, :, 0] = vis[0, :, 3] = s / 2
    return vis


def pin_p11_online_thresholds(seed=12):
    """P11: online per-stream SK thresholds (the build's rule for the paper's future
    work, see oracle/adaptive.py).

    (a) before n_warm clean windows nothing changes: outputs equal the fixed-threshold
        oracle's exactly;
    (b) with alpha = 0 the state is (count, mean tau, mean tau^2) over the windows the
        row did not flag -- the definition of a running mean, computed with numpy;
    (c) after warm-up a window is flagged iff tau leaves mean -/+ k sd of the earlier
        clean windows (numpy mean and population sd) or r exceeds gamma;
    (d) with alpha > 0, once n >= 1/alpha the mean relaxes geometrically: after N0
        windows at level A and k at level B, mean = tau_B + (1 - alpha)^k (mu0 - tau_B)."""
    from oracle import AdaptiveOracleStream
    rng = np.random.default_rng(seed)
    R, M, K, T, nblk = 12, 8, 32, 64, 6
    vis = (rng.standard_normal((R, T * nblk, 4)) + 1j * rng.standard_normal((R, T * nblk, 4))) / math.sqrt(2)
    vis[:, 100:120] *= 7.0
    vis[3, 200:260, :] = 3.0 * (1 + 1j)
    thr = dict(d=1.0, s_low=0.2, s_high=2.2, gamma=0.75, eps=EPS32)
    # (a)
    a = AdaptiveOracleStream(R, M, K, **thr, n_warm=10 ** 6)
    b = OracleStream(R, M, K, **thr)
    for k in range(nblk):
        oa, ob = a.process(vis[:, k * T:(k + 1) * T]), b.process(vis[:, k * T:(k + 1) * T])
        for key in ob:
            assert np.array_equal(oa[key], ob[key]), key
    # (b) and (c)
    st = AdaptiveOracleStream(R, M, K, **thr, alpha=0.0, k_sigma=2.5, n_warm=12)
    hist_tau = [[] for _ in range(R)]
    for k in range(nblk):
        lo_exp = np.full(R, thr["s_low"])
        hi_exp = np.full(R, thr["s_high"])
        for g in range(R):
            h = np.array(hist_tau[g])
            if h.size >= 12:
                lo_exp[g] = h.mean() - 2.5 * h.std()
                hi_exp[g] = h.mean() + 2.5 * h.std()
        out = st.process(vis[:, k * T:(k + 1) * T])
        assert np.allclose(out["s_low_used"], lo_exp, rtol=1e-12, atol=1e-12)
        assert np.allclose(out["s_high_used"], hi_exp, rtol=1e-12, atol=1e-12)
        exp = ~((out["tau"] >= lo_exp[:, None]) & (out["tau"] <= hi_exp[:, None])) | \
            (out["r_re"] > thr["gamma"]) | (out["r_im"] > thr["gamma"])
        assert np.array_equal(out["wflag"].astype(bool), exp)
        for g in range(R):
            hist_tau[g] += list(out["tau"][g][~out["wflag"][g].astype(bool)])
            h = np.array(hist_tau[g])
            n, mu, m2 = st.state[g]
            assert n == h.size
            if h.size:
                assert abs(mu - h.mean()) <= 1e-12 * max(1.0, abs(h.mean()))
                assert abs(m2 - (h * h).mean()) <= 1e-12 * max(1.0, (h * h).mean())
    assert any(f.any() for f in [st.thresholds()[0] != thr["s_low"]])   # warm-up was reached
    # (d)
    alpha, N0, kB = 1.0 / 8, 16, 11
    lead = (M * 1.0 + 1.0) / (M - 1.0)
    tau_B = lead * (M * 5.0 * M / ((2.0 * M) ** 2 + EPS32) - 1.0)
    v = _level_windows(["A"] * N0 + ["B"] * kB, M)
    st = AdaptiveOracleStream(1, M, M, 1.0, -1e300, 1e300, 2.0, EPS32, alpha=alpha,
                              n_warm=10 ** 6)
    st.process(v[:, :N0 * M])
    mu0, m20 = st.state[0, 1], st.state[0, 2]
    st.process(v[:, N0 * M:])
    q = (1.0 - alpha) ** kB
    assert abs(st.state[0, 1] - (tau_B + q * (mu0 - tau_B))) <= 1e-13
    assert abs(st.state[0, 2] - (tau_B ** 2 + q * (m20 - tau_B ** 2))) <= 1e-13
    assert abs(tau_B - lead * (0.25 - EPS32 / (4.0 * M * M) * 1.25)) <= 1e-9


ALL_PINS.append(pin_p11_online_thresholds)


def pin_p12_symmetries(seed=13):
    """P12: transformations of the data that the method's definitions leave unchanged
    (Sec. 2: Stokes parameters; Sec. 2.1: SK of |I|; Sec. 2.2: directions of (q, u, v)).

    (a) permuting the samples inside a window: every statistic is a sum over the window;
    (b) swapping the two polarisation feeds (xx <-> yy, xy <-> yx): I stays, Q and V
        change sign, so tau and both r stay;
    (c) negating every correlation, and (e) conjugating every correlation: |I| stays and
        each part of (Q, U, V) changes signs component-wise, so tau and both r stay;
    (d) scaling every correlation by c > 0 with eps = 0: tau and r are homogeneous of
        degree 0 in the data;
    (f) multiplying every correlation by j: |I| stays, the Re and Im parts of (Q, U, V)
        trade places (up to sign), so r_Re and r_Im swap;
    (g) on heavy-tailed data 0 <= r < 1 and tau <= Wd + 1 (above 0 up to the eps term)."""
    rng = np.random.default_rng(seed)
    R, M, nw = 9, 8, 40
    vis = rng.standard_normal((R, M * nw, 4)) + 1j * rng.standard_normal((R, M * nw, 4))
    vis[2, 40:80] *= 6.0
    vis[5, 120:200, :] = (2.0 + 1j) * np.array([1.0, 0.3 - 0.2j, 0.3 + 0.2j, 0.1])
    vis[7, :, 1:3] *= 0.01

    def stats(v, eps=EPS32):
        out = OracleStream(R, M, M, 1.3, -1e300, 1e300, 1e300, eps).process(v)
        return out["tau"], out["r_re"], out["r_im"]

    def close(a, b, tol=1e-12):
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=tol, atol=tol), float(np.max(np.abs(x - y)))

    base = stats(vis)
    perm = vis.reshape(R, nw, M, 4)[:, :, rng.permutation(M)].reshape(R, M * nw, 4)
    close(stats(perm), base)                                            # (a)
    close(stats(vis[..., [3, 2, 1, 0]]), base)                          # (b)
    close(stats(-vis), base)                                            # (c)
    close(stats(np.conj(vis)), base)                                    # (e)
    b0 = stats(vis, eps=0.0)
    close(stats(4.0 * vis, eps=0.0), b0)                                # (d)
    close(stats(0.25 * vis, eps=0.0), b0)
    t, rr, ri = stats(1j * vis)                                         # (f)
    close((t, rr, ri), (base[0], base[2], base[1]))
    # (g) bounds on heavy-tailed data: r is the length of a mean of vectors of length
    # below 1 (triangle inequality), and Cauchy-Schwarz bounds tau as in P2
    heavy = vis * rng.standard_cauchy((R, M * nw, 1))
    t, rr, ri = stats(heavy)
    d, W = 1.3, M
    lead = (W * d + 1.0) / (W - 1.0)
    assert np.all((rr >= 0) & (rr < 1)) and np.all((ri >= 0) & (ri < 1))
    assert np.all(t <= W * d + 1.0) and np.all(t >= -lead * 1e-6)


ALL_PINS.append(pin_p12_symmetries)


def pin_p13_sliding_windows(seed=14):
    """P13: overlapping windows (the build's extension, oracle/sliding.py).

    (a) window w of hop H is window i of the non-overlapping method run on the stream
        from sample (w mod L) H on, i = w div L (L = M / H): statistics and window
        flags equal those of the (independently pinned) plain oracle exactly;
    (b) one strong spike at sample t0 in noise, with thresholds that only the spike's
        windows cross (tau = Wd+1 for them, P2): the flagged samples are exactly
        [w1 H, w2 H + M), w1 = max(0, ceil((t0 - M + 1) / H)), w2 = floor(t0 / H);
    (c) averages over those flags, by brute force (mean of the unflagged samples of each
        bin of K samples, weight n / K);
    (d) splitting the stream into blocks at multiples of H changes nothing, and each
        call reports its windows, flags from the first sample that became final and
        the bins that closed;
    (e) H = M is the plain method."""
    rng = np.random.default_rng(seed)
    for R, M, H, K, N in ((5, 8, 4, 16, 96), (4, 12, 3, 24, 96), (3, 8, 2, 8, 64)):
        L = M // H
        vis = rng.standard_normal((R, N, 4)) + 1j * rng.standard_normal((R, N, 4))
        vis[1, 20:30] *= 8.0
        vis[2, 40:52, :] = 3.0 * (1 + 1j)
        thr = (1.0, 0.3, 2.2, 0.7, EPS32)
        sl = oracle.SlidingOracleStream(R, M, H, K, *thr).process(vis)
        E = (N - M) // H + 1
        assert sl["tau"].shape == (R, E) and sl["first_sample"] == 0
        # (a)
        for j in range(L):
            n = ((N - j * H) // M) * M
            pl = OracleStream(R, M, M, *thr).process(vis[:, j * H:j * H + n])
            for key in ("tau", "r_re", "r_im", "wflag"):
                assert np.array_equal(sl[key][:, j::L], pl[key]), (M, H, j, key)
        # (d)
        for cuts in ((H, 5 * H), tuple(range(2 * H, N, 3 * H)), (M - H, M, M + H)):
            st = oracle.SlidingOracleStream(R, M, H, K, *thr)
            edges = (0,) + tuple(c for c in cuts if 0 < c < N) + (N,)
            parts = []
            for a, b in zip(edges[:-1], edges[1:]):
                nwin, f0 = st.windows_for(b - a)
                n_out = st.outputs_for(b - a)
                out = st.process(vis[:, a:b])
                assert out["tau"].shape[1] == nwin and out["avg"].shape[1] == n_out
                assert out["first_sample"] == f0
                parts.append(out)
            for key in ("tau", "r_re", "r_im", "wflag", "avg", "weight"):
                got = np.concatenate([p[key] for p in parts], axis=1)
                assert np.array_equal(got, sl[key]), (M, H, cuts, key)
            for r in range(R):
                bits = []
                for p in parts:
                    bits += _bits(p["flagbits"][r], p["tau"].shape[1] * H)
                assert bits == _bits(sl["flagbits"][r], E * H), (M, H, cuts, r)
        # (b), (c)
        for t0 in (0, 1, H, M - 1, M + H + 1, N - M - 1):
            d = 1.0
            v = (rng.standard_normal((1, N, 4)) + 1j * rng.standard_normal((1, N, 4))) * 0.1
            v[0, t0] = 1e6
            # clean windows: tau <= Wd + 1 - 1e-3 almost surely; the spike's: ~ Wd + 1;
            # gamma = 1 never flags (r <= 1, strict comparison)
            out = oracle.SlidingOracleStream(1, M, H, K, d, -1e300, M * d + 1 - 1e-3, 1.0,
                                             EPS32).process(v)
            w1, w2 = max(0, -((M - 1 - t0) // H)), t0 // H
            want = np.zeros(E * H, dtype=bool)
            want[w1 * H:min(w2 * H + M, E * H)] = True
            got = np.array(_bits(out["flagbits"][0], E * H), dtype=bool)
            assert np.array_equal(got, want), (M, H, t0)
            n_bins = (E * H) // K
            for b in range(n_bins):
                keep = ~want[b * K:(b + 1) * K]
                x = v[0, b * K:(b + 1) * K][keep]
                mean = x.mean(axis=0) if keep.any() else np.zeros(4)
                ref = np.stack([mean.real, mean.imag], axis=-1).reshape(8)
                assert np.allclose(out["avg"][0, b], ref, rtol=1e-12, atol=1e-15), (M, H, t0, b)
                assert out["weight"][0, b] == keep.sum() / K
    # (e)
    R, M, K, N = 4, 8, 16, 64
    vis = rng.standard_normal((R, N, 4)) + 1j * rng.standard_normal((R, N, 4))
    vis[0, 8:16] *= 10.0
    thr = (1.0, 0.3, 2.2, 0.7, EPS32)
    a = oracle.SlidingOracleStream(R, M, M, K, *thr).process(vis)
    b = OracleStream(R, M, K, *thr).process(vis)
    for key in ("tau", "r_re", "r_im", "wflag", "flagbits", "avg", "weight"):
        assert np.array_equal(a[key], b[key]), key


ALL_PINS.append(pin_p13_sliding_windows)


def pin_p6b_given_window_flags(seed=16):
    """P6b: with window flags given by the caller (the flags of another arithmetic), the
    flag bits and averages follow those flags: mean of the samples of unflagged windows
    (numpy), weight n/K, bits over the flagged windows' samples; giving the oracle its
    own flags changes nothing."""
    rng = np.random.default_rng(seed)
    for M, K, T, F in ((4, 8, 24, 1), (5, 10, 20, 2), (16, 32, 64, 1)):
        R = 6 * F
        v = rng.standard_normal((R, T, 4)) + 1j * rng.standard_normal((R, T, 4))
        v[:, :M] *= 4.0
        thr = (1.0, 0.3, 2.0, 0.5, EPS32)
        own = OracleStream(R, M, K, *thr, F=F).process(v)
        again = OracleStream(R, M, K, *thr, F=F).process(v, wflag=own["wflag"])
        for k in own:
            assert np.array_equal(own[k], again[k]), k
        given = rng.integers(0, 2, size=(R // F, T // M)).astype(np.uint8)
        out = OracleStream(R, M, K, *thr, F=F).process(v, wflag=given)
        assert np.array_equal(out["wflag"], given)
        for row in range(R):
            keep = ~np.repeat(given[row // F], M).astype(bool)
            for b in range(T // K):
                sl = slice(b * K, (b + 1) * K)
                x, kp = v[row, sl], keep[sl]
                n = kp.sum()
                want = x[kp].mean(axis=0) if n else np.zeros(4)
                got = out["avg"][row, b].reshape(4, 2)
                assert np.allclose(got[:, 0], want.real, rtol=1e-13, atol=1e-14)
                assert np.allclose(got[:, 1], want.imag, rtol=1e-13, atol=1e-14)
                assert out["weight"][row, b] == n / K
            assert _bits(out["flagbits"][row], T) == [int(not k) for k in keep]


ALL_PINS.append(pin_p6b_given_window_flags)
