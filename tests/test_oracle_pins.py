"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a library routine (numpy / scipy), a generic optimiser applied to the
problem as the paper poses it, exhaustive search, a textbook error-rate
formula or an invariant.  None of them re-types the oracle's own formula.
"""
import math

import numpy as np
import pytest
from scipy import optimize
from scipy.sparse.linalg import cg as scipy_cg

import oracle
import synth


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ---------------------------------------------------------------------------
# Alphabet and slicer (Sec. II-A Gray mapping; Sec. III-A hard detection)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("M", [4, 16, 64])
def test_alphabet_unit_energy_and_gray_neighbours(M):
    pts = synth.qam_alphabet(M)
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-12
    a = math.sqrt(3.0 / (2.0 * (M - 1)))
    d = np.abs(pts[:, None] - pts[None, :])
    nn = np.isclose(d, 2 * a)  # horizontally / vertically adjacent points
    for i, j in zip(*np.nonzero(nn)):
        assert bin(i ^ j).count("1") == 1  # Gray: neighbours differ in one bit


@pytest.mark.parametrize("M", [4, 16, 64])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_slicer_inverts_alphabet(M, dtype):
    labels = np.arange(M, dtype=np.uint8)
    pts = synth.qam_alphabet(M)
    assert np.array_equal(oracle.slice_labels(pts, M, dtype=dtype), labels)
    assert np.allclose(oracle.label_points(labels, M), pts, atol=1e-15)


@pytest.mark.parametrize("M", [4, 16, 64])
def test_slicer_is_nearest_point(M):
    rng = np.random.default_rng(7)
    x = (rng.normal(size=4000) + 1j * rng.normal(size=4000)) * 1.3
    pts = synth.qam_alphabet(M)
    dist = np.abs(x[:, None] - pts[None, :])
    best = np.argmin(dist, axis=1)
    srt = np.sort(dist, axis=1)
    clear = (srt[:, 1] - srt[:, 0]) > 1e-9  # skip exact ties
    lab = oracle.slice_labels(x, M)
    assert np.array_equal(lab[clear], best[clear].astype(np.uint8))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_bpsk_alphabet_and_slicer(dtype):
    """M = 2 (BPSK, the alphabet of the real-segment prox): the points are
    -1 and +1, the slicer inverts them, picks the nearer point for any
    complex input (the imaginary part plays no role) and sends 0 to the
    lower level."""
    pts = synth.qam_alphabet(2)
    assert np.array_equal(pts, np.array([-1.0 + 0j, 1.0 + 0j]))
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-15
    assert np.array_equal(oracle.slice_labels(pts, 2, dtype=dtype), np.array([0, 1], dtype=np.uint8))
    assert np.array_equal(oracle.label_points(np.array([0, 1]), 2), pts)
    rng = np.random.default_rng(17)
    x = (rng.normal(size=3000) + 1j * rng.normal(size=3000)) * 1.5
    dist = np.abs(x[:, None] - pts[None, :])
    clear = np.abs(dist[:, 0] - dist[:, 1]) > 1e-9
    assert np.array_equal(oracle.slice_labels(x, 2, dtype=dtype)[clear], np.argmin(dist, axis=1)[clear])
    assert oracle.slice_labels(np.array([0.0 + 5j]), 2, dtype=dtype)[0] == 0
    assert oracle.box_radius(2) == 1.0


def test_slicer_ties_go_to_lower_level_and_clamp():
    M = 16
    a = math.sqrt(3.0 / (2.0 * (M - 1)))
    pts = synth.qam_alphabet(M)
    # boundaries at -2a, 0, 2a on each axis; values far outside clamp
    for xr, want_r in [(-2 * a, -3 * a), (0.0, -a), (2 * a, a), (50.0, 3 * a), (-50.0, -3 * a)]:
        lab = oracle.slice_labels(np.array([xr + 1j * a]), M)[0]
        p = pts[lab]
        assert abs(p.real - want_r) < 1e-12 and abs(p.imag - a) < 1e-12


# ---------------------------------------------------------------------------
# Helpers: problems drawn with the shared generator
# ---------------------------------------------------------------------------

def _ul(W=3, N=2, B=32, U=4, M=4, snr=10.0, seed=0):
    return synth.uplink_frame(W, N, B, U, M, snr, seed)


def _lmmse_numpy(H, y, delta):
    """(H^H H + delta I)^{-1} H^H y per subcarrier with numpy.linalg.solve."""
    W, B, U = H.shape
    out = np.empty((W, y.shape[1], U), dtype=complex)
    for w in range(W):
        G = H[w].conj().T @ H[w] + delta * np.eye(U)
        out[w] = np.linalg.solve(G, H[w].conj().T @ y[w].T).T
    return out


# ---------------------------------------------------------------------------
# Centralized references (Sec. III-A, Sec. IV-A)
# ---------------------------------------------------------------------------

def test_lmmse_and_zf_match_numpy():
    f = _ul(B=16, U=6)
    assert _rel(oracle.lmmse_ul(f["H"], f["y"], f["N0"]), _lmmse_numpy(f["H"], f["y"], f["N0"])) < 1e-12
    ls = np.stack([np.linalg.lstsq(f["H"][w], f["y"][w].T, rcond=None)[0].T for w in range(3)])
    assert _rel(oracle.lmmse_ul(f["H"], f["y"], 0.0), ls) < 1e-12


def test_zf_precoder_is_minimum_norm_solution():
    d = synth.downlink_frame(3, 2, 24, 5, 16, 3)
    x = oracle.zf_dl(d["H"], d["s"])
    for w in range(3):
        Hd = d["H"][w].T
        ref = (np.linalg.pinv(Hd) @ d["s"][w].T).T
        assert _rel(x[w], ref) < 1e-12


# ---------------------------------------------------------------------------
# Alg. 1 (decentralized ADMM detection)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("C", [1, 2, 4])
def test_admm_T1_closed_form(C):
    """T_max = 1: s = (N0/(rho Es) + C)^{-1} sum_c (H_c^H H_c + rho I)^{-1} H_c^H y_c."""
    f = _ul(B=32, U=4)
    rho = 1.7
    s = oracle.admm_ul(f["H"], f["y"], C=C, rho=rho, N0=f["N0"], T_max=1)
    S = 32 // C
    for w in range(3):
        acc = np.zeros((f["N"], 4), dtype=complex)
        for c in range(C):
            Hc = f["H"][w, c * S:(c + 1) * S]
            G = Hc.conj().T @ Hc + rho * np.eye(4)
            acc += np.linalg.solve(G, Hc.conj().T @ f["y"][w, :, c * S:(c + 1) * S].T).T
        assert _rel(s[w], acc / (f["N0"] / rho + C)) < 1e-13


@pytest.mark.parametrize("C", [1, 2, 4, 8])
@pytest.mark.parametrize("rho", [0.5, 1.0, 4.0])
def test_admm_converges_to_lmmse(C, rho):
    """(E0') is equivalent to (E0): converged ADMM equals the LMMSE solution."""
    f = _ul()
    s = oracle.admm_ul(f["H"], f["y"], C=C, rho=rho, N0=f["N0"], T_max=1500)
    assert _rel(s, _lmmse_numpy(f["H"], f["y"], f["N0"])) < 1e-10


@pytest.mark.parametrize("C", [1, 4])
def test_admm_zf_converges_to_least_squares(C):
    f = _ul()
    s = oracle.admm_ul(f["H"], f["y"], C=C, rho=1.0, N0=f["N0"], T_max=1500, reg=oracle.REG_ZF)
    assert _rel(s, _lmmse_numpy(f["H"], f["y"], 0.0)) < 1e-10


@pytest.mark.parametrize("B,C,U", [(32, 4, 4), (32, 2, 16), (32, 8, 4), (24, 6, 8)])
@pytest.mark.parametrize("T", [1, 2, 3, 5])
def test_admm_modes_identical(B, C, U, T):
    """(E1) closed form and its Woodbury (S x S) variant give the same iterates."""
    f = _ul(B=B, U=U, M=16, seed=B + C + U)
    a = oracle.admm_ul(f["H"], f["y"], C=C, rho=0.8, N0=f["N0"], T_max=T, mode=oracle.MODE_UXU)
    b = oracle.admm_ul(f["H"], f["y"], C=C, rho=0.8, N0=f["N0"], T_max=T, mode=oracle.MODE_SXS)
    assert _rel(a, b) < 1e-12


def _admm_generic(H, y, C, rho, gamma, T, prox):
    """ADMM of Sec. III-B in its own order (E1), (E2), (E3), each step solved
    by a generic solver: (E1) as the stacked least-squares problem, (E2) by the
    caller's generic minimiser of g(s) + sum_c rho/2 ||s - z_c - lambda_c||^2."""
    B, U = H.shape
    S = B // C
    s = np.zeros(U, dtype=complex)
    lam = [np.zeros(U, dtype=complex) for _ in range(C)]
    for _ in range(T):
        z = []
        for c in range(C):
            A = np.vstack([H[c * S:(c + 1) * S], math.sqrt(rho) * np.eye(U)])
            b = np.concatenate([y[c * S:(c + 1) * S], math.sqrt(rho) * (s - lam[c])])
            z.append(np.linalg.lstsq(A, b, rcond=None)[0])
        s_new = prox([z[c] + lam[c] for c in range(C)])
        lam = [lam[c] - gamma * (s_new - z[c]) for c in range(C)]
        s = s_new
    return s


def _prox_quadratic(rho, g_weight):
    """argmin g_weight/2 ||s||^2 + sum_c rho/2 ||s - w_c||^2 by stacked lstsq."""
    def prox(ws):
        U = ws[0].size
        blocks = [math.sqrt(rho) * np.eye(U) for _ in ws]
        rhs = [math.sqrt(rho) * wc for wc in ws]
        if g_weight > 0:
            blocks.insert(0, math.sqrt(g_weight) * np.eye(U))
            rhs.insert(0, np.zeros(U))
        return np.linalg.lstsq(np.vstack(blocks), np.concatenate(rhs), rcond=None)[0]
    return prox


def _prox_box(rho, r):
    """argmin_{|Re s|,|Im s| <= r} sum_c rho/2 ||s - w_c||^2 by bounded lstsq."""
    def prox(ws):
        U = ws[0].size
        A = np.vstack([math.sqrt(rho) * np.eye(2 * U) for _ in ws])
        b = np.concatenate([math.sqrt(rho) * np.concatenate([wc.real, wc.imag]) for wc in ws])
        sol = optimize.lsq_linear(A, b, bounds=(-r, r), method="bvls", tol=1e-14).x
        return sol[:U] + 1j * sol[U:]
    return prox


def _prox_bpsk(rho, r):
    """argmin over real s with |s| <= r of sum_c rho/2 ||s - w_c||^2 by bounded
    lstsq (the imaginary parts of w_c only add a constant)."""
    def prox(ws):
        U = ws[0].size
        A = np.vstack([math.sqrt(rho) * np.eye(U) for _ in ws])
        b = np.concatenate([math.sqrt(rho) * wc.real for wc in ws])
        return optimize.lsq_linear(A, b, bounds=(-r, r), method="bvls", tol=1e-14).x + 0j
    return prox


@pytest.mark.parametrize("reg", ["mmse", "zf", "box", "bpsk"])
@pytest.mark.parametrize("T", [1, 2, 3, 5])
def test_admm_matches_generic_steps(reg, T):
    """Alg. 1 (steps reordered E3, E1, E2; T_max counts E1/E2 passes) equals
    Sec. III-B's ADMM solved step by step with generic solvers."""
    f = _ul(W=2, N=2, B=24, U=4, M=2 if reg == "bpsk" else 16, snr=6.0, seed=11)
    C, rho, gamma = 3, 0.9, 1.0
    r = oracle.box_radius(2 if reg == "bpsk" else 16)
    if reg == "mmse":
        prox, code = _prox_quadratic(rho, f["N0"] / f["Es"]), oracle.REG_MMSE
    elif reg == "zf":
        prox, code = _prox_quadratic(rho, 0.0), oracle.REG_ZF
    elif reg == "bpsk":
        prox, code = _prox_bpsk(rho, r), oracle.REG_BPSK
    else:
        prox, code = _prox_box(rho, r), oracle.REG_BOX
    s = oracle.admm_ul(f["H"], f["y"], C=C, rho=rho, N0=f["N0"], T_max=T, gamma=gamma,
                       reg=code, box_r=r)
    for w in range(2):
        for n in range(2):
            ref = _admm_generic(f["H"][w], f["y"][w, n], C, rho, gamma, T, prox)
            assert np.abs(s[w, n] - ref).max() < 1e-10


@pytest.mark.parametrize("reg", ["box", "bpsk"])
@pytest.mark.parametrize("C", [1, 4])
def test_admm_constrained_converges_to_bounded_least_squares(reg, C):
    """With g the indicator of the box (E2-BOX) or of the real segment (BPSK),
    (E0) is least squares under bounds: converged ADMM equals scipy's
    bounded-variable least squares on the real form of y = H s, and some
    bounds are active (the constraint does work at this SNR)."""
    M = 2 if reg == "bpsk" else 4
    f = _ul(W=2, N=3, B=16, U=4, M=M, snr=3.0, seed=23 + C)
    r = oracle.box_radius(M)
    s = oracle.admm_ul(f["H"], f["y"], C=C, rho=1.0, N0=f["N0"], T_max=4000,
                       reg=oracle.REG_BPSK if reg == "bpsk" else oracle.REG_BOX, box_r=r)
    active = 0
    for w in range(2):
        H = f["H"][w]
        if reg == "bpsk":   # s real: [Re H; Im H] s = [Re y; Im y]
            A = np.vstack([H.real, H.imag])
        else:               # s = a + ib: [[Re H, -Im H], [Im H, Re H]] (a, b)
            A = np.block([[H.real, -H.imag], [H.imag, H.real]])
        for n in range(3):
            y = f["y"][w, n]
            sol = optimize.lsq_linear(A, np.concatenate([y.real, y.imag]), bounds=(-r, r),
                                      method="bvls", tol=1e-14).x
            ref = sol + 0j if reg == "bpsk" else sol[:4] + 1j * sol[4:]
            assert np.abs(s[w, n] - ref).max() < 1e-8
            active += int(np.sum(np.abs(sol) > r - 1e-12))
    assert active > 0
    if reg == "bpsk":
        assert np.all(s.imag == 0.0)


@pytest.mark.parametrize("algo", ["admm_mmse", "admm_zf", "dl"])
def test_linearity(algo):
    """MMSE/ZF ADMM detection and eps = 0 beamforming are linear maps of y / s."""
    f1 = _ul(seed=1, M=16)
    f2 = _ul(seed=2, M=16)
    a = 0.7 - 1.3j
    if algo == "dl":
        fn = lambda v: oracle.admm_dl(f1["H"], v, C=4, rho=0.6, T_max=4)
        v1, v2 = f1["s"], f2["s"]
    else:
        reg = oracle.REG_MMSE if algo == "admm_mmse" else oracle.REG_ZF
        fn = lambda v: oracle.admm_ul(f1["H"], v, C=4, rho=0.6, N0=f1["N0"], T_max=4, reg=reg)
        v1, v2 = f1["y"], f2["y"]
    assert _rel(fn(a * v1 + v2), a * fn(v1) + fn(v2)) < 1e-12


# ---------------------------------------------------------------------------
# Alg. 2 (decentralized CG detection)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("C", [1, 2, 4, 8])
def test_cg_exact_after_U_steps(C):
    f = _ul(B=32, U=4, snr=15.0, seed=5)
    x = oracle.cg_ul(f["H"], f["y"], C=C, rho=f["N0"], T_max=4)
    assert _rel(x, _lmmse_numpy(f["H"], f["y"], f["N0"])) < 1e-9


@pytest.mark.parametrize("T", [1, 2, 3, 5])
def test_cg_matches_library_cg(T):
    """Finite-T iterates equal scipy's CG on (H^H H + rho I) x = H^H y, x0 = 0."""
    f = _ul(W=2, N=3, B=32, U=6, M=16, seed=9)
    rho = f["N0"]
    x = oracle.cg_ul(f["H"], f["y"], C=4, rho=rho, T_max=T)
    for w in range(2):
        A = f["H"][w].conj().T @ f["H"][w] + rho * np.eye(6)
        for n in range(3):
            b = f["H"][w].conj().T @ f["y"][w, n]
            ref, _ = scipy_cg(A, b, x0=np.zeros(6, dtype=complex), rtol=0.0, atol=0.0, maxiter=T)
            assert np.abs(x[w, n] - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())


def test_cg_invariant_to_cluster_count():
    f = _ul(W=2, N=2, B=32, U=8, M=16, seed=4)
    xs = [oracle.cg_ul(f["H"], f["y"], C=C, rho=f["N0"], T_max=3) for C in (1, 2, 4, 8, 16)]
    for x in xs[1:]:
        assert _rel(x, xs[0]) < 1e-12


def test_cg_homogeneous():
    f = _ul(seed=8, M=16)
    a = -0.4 + 2.2j
    x1 = oracle.cg_ul(f["H"], f["y"], C=4, rho=f["N0"], T_max=2)
    x2 = oracle.cg_ul(f["H"], a * f["y"], C=4, rho=f["N0"], T_max=2)
    assert _rel(x2, a * x1) < 1e-12


def test_cg_zero_input_stops():
    f = _ul()
    x = oracle.cg_ul(f["H"], np.zeros_like(f["y"]), C=2, rho=0.0, T_max=3)
    assert np.all(x == 0)


# ---------------------------------------------------------------------------
# Alg. 3 (decentralized ADMM beamforming)
# ---------------------------------------------------------------------------

def _dl(W=2, N=2, B=24, U=4, M=16, seed=3):
    return synth.downlink_frame(W, N, B, U, M, seed)


@pytest.mark.parametrize("C", [1, 2, 4])
def test_dl_converges_to_zf(C):
    d = _dl(B=32, U=4)
    x = oracle.admm_dl(d["H"], d["s"], C=C, rho=1.0, T_max=1500)
    ref = oracle.zf_dl(d["H"], d["s"])
    assert _rel(x, ref) < 1e-9
    for w in range(2):
        assert np.abs(d["H"][w].T @ x[w].T - d["s"][w].T).max() < 1e-9


@pytest.mark.parametrize("B,C,U", [(32, 4, 4), (32, 2, 16), (24, 6, 8)])
def test_dl_T1_closed_form(B, C, U):
    d = _dl(B=B, U=U, seed=B + U)
    rho = 0.7
    x = oracle.admm_dl(d["H"], d["s"], C=C, rho=rho, T_max=1)
    S = B // C
    k = max(U / B, 1.0 / C)
    for w in range(2):
        for c in range(C):
            Hd = d["H"][w, c * S:(c + 1) * S].T
            A = Hd.conj().T @ Hd + np.eye(S) / rho
            ref = np.linalg.solve(A, Hd.conj().T @ (k * d["s"][w].T)).T
            assert _rel(x[w, :, c * S:(c + 1) * S], ref) < 1e-12


@pytest.mark.parametrize("B,C,U", [(32, 4, 4), (32, 2, 16), (24, 6, 8)])
@pytest.mark.parametrize("T", [1, 2, 4])
def test_dl_modes_identical(B, C, U, T):
    d = _dl(B=B, U=U, seed=2 * B + U)
    a = oracle.admm_dl(d["H"], d["s"], C=C, rho=1.3, T_max=T, mode=oracle.MODE_UXU)
    b = oracle.admm_dl(d["H"], d["s"], C=C, rho=1.3, T_max=T, mode=oracle.MODE_SXS)
    assert _rel(a, b) < 1e-12


def _dl_generic(H, s, C, rho, gamma, T, eps):
    """ADMM of Sec. IV-B in its own order (P1), (P2), (P3) with generic
    solvers: (P1) as stacked least squares, (P2) as the projection of
    w_all onto {z : ||s - sum_c z_c|| <= eps} (KKT system for eps = 0, SLSQP
    otherwise)."""
    B, U = H.shape
    S = B // C
    Hd = [H[c * S:(c + 1) * S].T for c in range(C)]
    z = [max(U / B, 1.0 / C) * s for _ in range(C)]
    lam = [np.zeros(U, dtype=complex) for _ in range(C)]
    for t in range(T):
        x = []
        for c in range(C):
            A = np.vstack([math.sqrt(rho) * Hd[c], np.eye(S)])
            b = np.concatenate([math.sqrt(rho) * (z[c] + lam[c]), np.zeros(S)])
            x.append(np.linalg.lstsq(A, b, rcond=None)[0])
        if t == T - 1:
            return np.concatenate(x)
        wall = np.concatenate([Hd[c] @ x[c] - lam[c] for c in range(C)])
        D = np.kron(np.ones((1, C)), np.eye(U))
        if eps == 0.0:
            K = np.block([[np.eye(U * C), D.conj().T], [D, np.zeros((U, U))]])
            zall = np.linalg.solve(K, np.concatenate([wall, s]))[:U * C]
        else:
            Dr = np.block([[D, np.zeros_like(D)], [np.zeros_like(D), D]]).real
            wr = np.concatenate([wall.real, wall.imag])
            sr = np.concatenate([s.real, s.imag])
            cons = {"type": "ineq", "fun": lambda v: eps ** 2 - np.sum((sr - Dr @ v) ** 2)}
            res = optimize.minimize(lambda v: 0.5 * np.sum((v - wr) ** 2), wr,
                                    jac=lambda v: v - wr, constraints=[cons],
                                    method="SLSQP", options={"ftol": 1e-15, "maxiter": 500})
            zall = res.x[:U * C] + 1j * res.x[U * C:]
        znew = [zall[c * U:(c + 1) * U] for c in range(C)]
        lam = [lam[c] - gamma * (Hd[c] @ x[c] - znew[c]) for c in range(C)]
        z = znew


@pytest.mark.parametrize("T", [1, 2, 3, 5])
def test_dl_matches_generic_steps(T):
    """Alg. 3 (steps reordered P2, P3, P1) equals Sec. IV-B's ADMM."""
    d = _dl(W=2, N=2, B=24, U=4, seed=21)
    x = oracle.admm_dl(d["H"], d["s"], C=3, rho=1.4, T_max=T)
    for w in range(2):
        for n in range(2):
            ref = _dl_generic(d["H"][w], d["s"][w, n], 3, 1.4, 1.0, T, 0.0)
            assert np.abs(x[w, n] - ref).max() < 1e-10


@pytest.mark.parametrize("T", [2, 3])
def test_dl_eps_projection_matches_generic(T):
    """Lemma 2 with eps > 0 equals a generic constrained projection."""
    d = _dl(W=1, N=2, B=16, U=4, seed=33)
    eps = 0.3
    x = oracle.admm_dl(d["H"], d["s"], C=2, rho=1.0, T_max=T, eps=eps)
    for n in range(2):
        ref = _dl_generic(d["H"][0], d["s"][0, n], 2, 1.0, 1.0, T, eps)
        assert np.abs(x[0, n] - ref).max() < 1e-5


# ---------------------------------------------------------------------------
# Detection quality: brute-force ML, ZF error-rate closed form
# ---------------------------------------------------------------------------

def test_ml_bruteforce_tiny_qpsk_high_snr():
    f = synth.uplink_frame(W=20, N=2, B=8, U=3, M=4, snr_db=30.0, seed=41)
    lab_lmmse = oracle.slice_labels(oracle.lmmse_ul(f["H"], f["y"], f["N0"]), 4)
    lab_admm = oracle.slice_labels(
        oracle.admm_ul(f["H"], f["y"], C=2, rho=1.0, N0=f["N0"], T_max=5), 4)
    lab_cg = oracle.slice_labels(oracle.cg_ul(f["H"], f["y"], C=2, rho=f["N0"], T_max=3), 4)
    for w in range(20):
        for n in range(2):
            ml = oracle.ml_detect(f["H"][w], f["y"][w, n], 4)
            assert np.array_equal(ml, f["labels"][w, n])
    for lab in (lab_lmmse, lab_admm, lab_cg):
        assert np.array_equal(lab, f["labels"])


def test_ml_not_worse_than_lmmse_low_snr():
    f = synth.uplink_frame(W=150, N=2, B=4, U=3, M=4, snr_db=4.0, seed=42)
    lab_lmmse = oracle.slice_labels(oracle.lmmse_ul(f["H"], f["y"], f["N0"]), 4)
    err_ml = err_lin = 0
    for w in range(150):
        for n in range(2):
            ml = oracle.ml_detect(f["H"][w], f["y"][w, n], 4)
            err_ml += int(not np.array_equal(ml, f["labels"][w, n]))
            err_lin += int(not np.array_equal(lab_lmmse[w, n], f["labels"][w, n]))
    assert err_ml <= err_lin and err_lin > 0


def test_zf_qpsk_ber_matches_rayleigh_closed_form():
    """ZF on i.i.d. Rayleigh: per-user post-equaliser SNR is Gamma(L) with
    L = B - U + 1, so the QPSK bit error rate is that of BPSK with L-branch
    maximum-ratio combining (Proakis), mean branch SNR Es / (2 N0)."""
    B, U, snr = 4, 2, 10.0
    f = synth.uplink_frame(W=50000, N=4, B=B, U=U, M=4, snr_db=snr, seed=43)
    lab = oracle.slice_labels(oracle.lmmse_ul(f["H"], f["y"], 0.0), 4)
    nbits = lab.size * 2
    ber = oracle.bit_errors(lab, f["labels"]) / nbits
    L = B - U + 1
    g = f["Es"] / (2.0 * f["N0"])
    mu = math.sqrt(g / (1.0 + g))
    pb = ((1 - mu) / 2) ** L * sum(math.comb(L - 1 + k, k) * ((1 + mu) / 2) ** k for k in range(L))
    sigma = math.sqrt(pb * (1 - pb) / nbits)
    assert abs(ber - pb) < 4.0 * sigma, (ber, pb, sigma)


# ---------------------------------------------------------------------------
# Argument checks
# ---------------------------------------------------------------------------

def test_oracle_rejects_bad_arguments():
    f = _ul()
    with pytest.raises(ValueError):
        oracle.admm_ul(f["H"], f["y"], C=5, rho=1.0, N0=f["N0"])  # 32 % 5 != 0
    with pytest.raises(ValueError):
        oracle.admm_ul(f["H"], f["y"], C=2, rho=0.0, N0=f["N0"])
    with pytest.raises(ValueError):
        oracle.admm_ul(f["H"], f["y"], C=2, rho=1.0, N0=f["N0"], T_max=0)
    with pytest.raises(ValueError):
        oracle.admm_dl(f["H"], f["s"], C=2, rho=1.0, eps=-1.0)


# ---------------------------------------------------------------------------
# Soft outputs: LLR statistics of the linear estimate and max-log LLRs
# ---------------------------------------------------------------------------

def test_llr_qpsk_closed_form():
    """QPSK: per axis the two points are +-a (a = 1/sqrt 2) with Gray bit 1 on
    the positive point, so L = ((x - mu a)^2 - (x + mu a)^2) / nu^2 = -4 mu a x / nu^2."""
    rng = np.random.default_rng(11)
    x = rng.normal(size=(3, 5, 2)) + 1j * rng.normal(size=(3, 5, 2))
    mu = rng.uniform(0.3, 1.0, size=(3, 2))
    nu2 = rng.uniform(0.05, 2.0, size=(3, 2))
    L = oracle.llr_maxlog(x, mu, nu2, 4)
    a = 1.0 / math.sqrt(2.0)
    np.testing.assert_allclose(L[..., 0], -4 * mu[:, None, :] * a * x.real / nu2[:, None, :], rtol=1e-12)
    np.testing.assert_allclose(L[..., 1], -4 * mu[:, None, :] * a * x.imag / nu2[:, None, :], rtol=1e-12)


@pytest.mark.parametrize("M", [4, 16, 64, 256])
def test_llr_signs_are_the_hard_decisions(M):
    """The max-log decision of each bit (L < 0: bit 1) is the bit of the
    nearest point to x / mu, i.e. the slicer's label of x / mu."""
    rng = np.random.default_rng(M)
    x = 1.3 * (rng.normal(size=(4, 6, 3)) + 1j * rng.normal(size=(4, 6, 3)))
    mu = rng.uniform(0.5, 1.0, size=(4, 3))
    nu2 = rng.uniform(0.1, 1.0, size=(4, 3))
    L = oracle.llr_maxlog(x, mu, nu2, M)
    lab = oracle.slice_labels(x / mu[:, None, :], M).astype(np.int64)
    m = L.shape[-1]
    for j in range(m):
        bit = (lab >> (m - 1 - j)) & 1
        clear = np.abs(L[..., j]) > 1e-9
        assert np.array_equal((L[..., j] < 0)[clear], (bit == 1)[clear])


@pytest.mark.parametrize("M", [16, 64])
def test_llr_reflection_flips_only_the_axis_msb(M):
    """Binary-reflected Gray code: reflecting a PAM index flips only its top
    bit, so x -> -conj(x) (real axis reflected) negates the first LLR and
    leaves the other real-axis LLRs unchanged."""
    rng = np.random.default_rng(7)
    x = rng.normal(size=(2, 3, 4)) + 1j * rng.normal(size=(2, 3, 4))
    mu = rng.uniform(0.5, 1.0, size=(2, 4))
    nu2 = rng.uniform(0.1, 1.0, size=(2, 4))
    L = oracle.llr_maxlog(x, mu, nu2, M)
    Lr = oracle.llr_maxlog(-np.conj(x), mu, nu2, M)
    half = L.shape[-1] // 2
    np.testing.assert_allclose(Lr[..., 0], -L[..., 0], atol=1e-12)
    np.testing.assert_allclose(Lr[..., 1:half], L[..., 1:half], atol=1e-12)
    np.testing.assert_allclose(Lr[..., half:], L[..., half:], atol=1e-12)


def test_llr_stats_zf_orthogonal_columns():
    """ZF with orthogonal columns of norm^2 b: A = I / b, mu = 1, nu^2 = N0 / b."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(16, 4)) + 1j * rng.normal(size=(16, 4)))
    H = (math.sqrt(5.0) * Q)[None]
    mu, nu2 = oracle.llr_stats(H, N0=0.3, reg=oracle.REG_ZF)
    np.testing.assert_allclose(mu, 1.0, rtol=1e-13)
    np.testing.assert_allclose(nu2, 0.3 / 5.0, rtol=1e-12)


def test_llr_stats_mmse_monte_carlo():
    """The LMMSE estimate of a fixed channel: over many symbol and noise draws,
    E[x_u conj(s_u)] / Es -> mu_u and E|x_u - mu_u s_u|^2 -> nu_u^2."""
    rng = np.random.default_rng(5)
    B, U, M, N0 = 12, 4, 16, 0.8
    H = (rng.normal(size=(B, U)) + 1j * rng.normal(size=(B, U))) / math.sqrt(2.0)
    mu, nu2 = oracle.llr_stats(H[None], N0=N0, Es=1.0, reg=oracle.REG_MMSE)
    K = 200000
    s = oracle.label_points(rng.integers(0, M, size=(K, U)), M)
    n = math.sqrt(N0 / 2) * (rng.normal(size=(K, B)) + 1j * rng.normal(size=(K, B)))
    y = s @ H.T + n
    A = np.linalg.inv(H.conj().T @ H + N0 * np.eye(U))
    x = y @ (A @ H.conj().T).T
    mu_emp = np.mean(x * s.conj(), axis=0).real
    nu2_emp = np.mean(np.abs(x - mu[0] * s) ** 2, axis=0)
    np.testing.assert_allclose(mu_emp, mu[0], rtol=0.01)
    np.testing.assert_allclose(nu2_emp, nu2[0], rtol=0.03)


def test_synth_at_snr_keeps_channel_and_symbols():
    """synth.at_snr: same H and transmitted symbols, y - H s has the noise
    variance of the requested SNR (N0 = U Es / SNR)."""
    f = synth.uplink_frame(80, 14, 16, 4, 16, 10.0, seed=11)
    g = synth.at_snr(f, 25.0, seed=12)
    assert np.array_equal(g["H"], f["H"]) and np.array_equal(g["labels"], f["labels"])
    n = g["y"] - np.einsum("wbu,wnu->wnb", f["H"], f["s"])
    N0 = 4 * 1.0 / 10 ** 2.5
    assert abs(g["N0"] - N0) < 1e-15
    assert abs(np.mean(np.abs(n) ** 2) / N0 - 1.0) < 0.02
