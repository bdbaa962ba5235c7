"""Pins of the FP64 oracle to facts fixed by the mathematics, not by the oracle.

Each test states the fact it checks.  Together they are chosen so that a
dropped term, a wrong sign, a swapped a/c direction, a b-term on the wrong
axis pair, a transposed operand, a residual taken from the wrong state or a
Gauss-Seidel (in-place) update would fail at least one of them.
"""
import numpy as np
import pytest

import jacobi_inputs as ji

OMEGA = 0.8


def const_fields(I, J, K, alphas, b=None, wrk1=None, rng=None):
    """a_d = c_d = alphas[d] everywhere, a3 = 1/(2 sum alphas)."""
    shape = (K, J, I)
    f = {}
    for d, (a, c) in enumerate((("a0", "c0"), ("a1", "c1"), ("a2", "c2"))):
        f[a] = np.full(shape, float(alphas[d]))
        f[c] = np.full(shape, float(alphas[d]))
    for q, name in enumerate(("b0", "b1", "b2")):
        f[name] = np.zeros(shape) if b is None else b[q]
    f["wrk1"] = np.zeros(shape) if wrk1 is None else wrk1
    f["a3"] = np.full(shape, 1.0 / (2.0 * sum(alphas)))
    f["bnd"] = ji.interior_mask(I, J, K)
    return f


def grid_coords(I, J, K):
    k, j, i = np.meshgrid(np.arange(K, dtype=float), np.arange(J, dtype=float),
                          np.arange(I, dtype=float), indexing="ij")
    return i, j, k


def interior(a):
    return a[1:-1, 1:-1, 1:-1]


# ---------------------------------------------------------------- fixed point
def test_constant_field_is_exact_fixed_point(oracle_mod):
    """a0=a1=a2=c0=1.5, c1=c2=1: S = 8 and a3 = 1/8 exactly; with wrk1 = 0 and
    p = 0.75 every product and sum is exact, so ss = 0 bitwise, p is unchanged
    and the residual is exactly 0, whatever the b coefficients are."""
    I, J, K = 9, 10, 11
    rng = np.random.default_rng(0)
    shape = (K, J, I)
    f = {n: np.full(shape, v) for n, v in (("a0", 1.5), ("a1", 1.5), ("a2", 1.5),
                                          ("c0", 1.5), ("c1", 1.0), ("c2", 1.0), ("a3", 0.125))}
    for n in ("b0", "b1", "b2"):
        f[n] = rng.uniform(-0.02, 0.02, shape)
    f["wrk1"] = np.zeros(shape)
    f["bnd"] = ji.interior_mask(I, J, K)
    f["p"] = np.full(shape, 0.75)
    p, g = oracle_mod.run(f, 7, OMEGA)
    assert np.array_equal(p, f["p"]) and g == 0.0


def test_random_coefficients_near_fixed_point(oracle_mod):
    """With the workload's random coefficients (a3 = 1/S) and wrk1 = 0, a
    constant field is a fixed point up to rounding: |ss| within a few ulp."""
    I, J, K = 8, 9, 10
    f = ji.himeno_fields(I, J, K)
    f["wrk1"] = np.zeros_like(f["wrk1"])
    p0 = np.full_like(f["p"], 0.5)
    p1, g = oracle_mod.sweep(f, p0, OMEGA)
    assert np.abs(p1 - p0).max() < 8 * np.finfo(float).eps
    assert g < (I * J * K) * (8 * np.finfo(float).eps) ** 2


# ---------------------------------------------------------- sine-mode decay
@pytest.mark.parametrize("alphas,modes,dims", [((1.0, 1.3, 0.7), (1, 2, 1), (17, 19, 23)),
                                               ((0.9, 1.1, 1.05), (3, 1, 2), (12, 9, 16))])
def test_sine_mode_decays_by_closed_form(oracle_mod, alphas, modes, dims):
    """a_d = c_d (constant per direction), b = 0, wrk1 = 0 and a discrete sine
    mode with zero faces: the stencil maps the mode to lambda times itself with
    lambda = sum a_d cos(theta_d) / sum a_d, so every sweep multiplies it by
    g = 1 - omega(1 - lambda) and the residual of sweep n is
    (1 - lambda)^2 g^(2(n-1)) sum_interior p0^2."""
    I, J, K = dims
    l, m, n_ = modes
    f = const_fields(I, J, K, alphas)
    i, j, k = grid_coords(I, J, K)
    th = (np.pi * l / (I - 1), np.pi * m / (J - 1), np.pi * n_ / (K - 1))
    p0 = np.sin(th[0] * i) * np.sin(th[1] * j) * np.sin(th[2] * k)
    p0 *= ji.interior_mask(I, J, K)                   # faces exactly zero
    f["p"] = p0
    lam = sum(a * np.cos(t) for a, t in zip(alphas, th)) / sum(alphas)
    g = 1.0 - OMEGA * (1.0 - lam)
    for n in (1, 2, 5, 13):
        p, gosa = oracle_mod.run(f, n, OMEGA)
        want = g ** n * p0
        assert np.abs(p - want).max() <= 1e-13 * np.abs(p0).max()
        gosa_want = (1 - lam) ** 2 * g ** (2 * (n - 1)) * np.sum(interior(p0) ** 2)
        assert abs(gosa - gosa_want) <= 1e-12 * gosa_want


# --------------------------------------------- directions and b-term pairs
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_field_pins_a_versus_c_direction(oracle_mod, axis):
    """p equal to the coordinate along one axis, random a, b, c, wrk1 and
    a3 = 1/S: the a (forward) and c (backward) neighbours differ by +-1, all
    b brackets vanish, so ss = a3 (a_d - c_d + wrk1) up to rounding."""
    I, J, K = 6, 7, 8
    f = ji.himeno_fields(I, J, K, seed=11)
    i, j, k = grid_coords(I, J, K)
    f["p"] = (i, j, k)[axis].copy()
    p1, _ = oracle_mod.sweep(f, f["p"], OMEGA)
    a, c = f["a%d" % axis], f["c%d" % axis]
    want = OMEGA * f["a3"] * (a - c + f["wrk1"])
    assert np.abs(interior(p1 - f["p"]) - interior(want)).max() < 1e-14


@pytest.mark.parametrize("pair,bname", [((0, 1), "b0"), ((1, 2), "b1"), ((0, 2), "b2")])
def test_bilinear_field_pins_cross_terms(oracle_mod, pair, bname):
    """p = x_u * x_v for one axis pair: its 4-point cross difference is exactly
    4 for that pair and 0 for the other two, and the a/c parts cancel
    (a_d = c_d).  With sum(alphas) = 4 every other operation is exact, so one
    sweep gives p' - p = omega/8 * (4 b + wrk1) with the b of that pair."""
    I, J, K = 7, 8, 9
    rng = np.random.default_rng(5)
    shape = (K, J, I)
    b = [rng.uniform(-0.02, 0.02, shape) for _ in range(3)]
    wrk1 = rng.uniform(-1e-3, 1e-3, shape)
    f = const_fields(I, J, K, (1.5, 1.25, 1.25), b=b, wrk1=wrk1)
    xyz = grid_coords(I, J, K)
    f["p"] = xyz[pair[0]] * xyz[pair[1]]
    p1, _ = oracle_mod.sweep(f, f["p"], OMEGA)
    want = OMEGA * 0.125 * (4.0 * f[bname] + wrk1)
    assert np.abs(interior(p1 - f["p"]) - interior(want)).max() < 4e-15 * I * J * K


# ------------------------------------------------------------ symmetries
def mirror(f, axis):
    """Reflect every array along one axis (i: numpy axis 2, j: 1, k: 0); the a
    and c coefficients of that axis swap and the two b brackets that contain
    the axis change sign."""
    nax = 2 - axis
    g = {n: np.flip(v, nax).copy() for n, v in f.items()}
    a, c = "a%d" % axis, "c%d" % axis
    g[a], g[c] = g[c], g[a]
    for bname, axes in (("b0", (0, 1)), ("b1", (1, 2)), ("b2", (0, 2))):
        if axis in axes:
            g[bname] = -g[bname]
    return g


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(oracle_mod, axis):
    f = ji.himeno_fields(7, 8, 9, seed=3)
    p, g = oracle_mod.run(f, 4, OMEGA)
    fm = mirror(f, axis)
    pm, gm = oracle_mod.run(fm, 4, OMEGA)
    assert np.abs(np.flip(pm, 2 - axis) - p).max() < 1e-14
    assert abs(gm - g) <= 1e-12 * g


def test_axis_swap_symmetry(oracle_mod):
    """Swapping the i and j axes swaps a0/a1, c0/c1 and the (j,k) and (i,k)
    cross coefficients b1/b2; b0's (i,j) bracket is symmetric."""
    f = ji.himeno_fields(7, 9, 8, seed=4)
    p, g = oracle_mod.run(f, 3, OMEGA)
    t = {n: np.ascontiguousarray(np.swapaxes(v, 1, 2)) for n, v in f.items()}
    t["a0"], t["a1"] = t["a1"], t["a0"]
    t["c0"], t["c1"] = t["c1"], t["c0"]
    t["b1"], t["b2"] = t["b2"], t["b1"]
    pt, gt = oracle_mod.run(t, 3, OMEGA)
    assert np.abs(np.swapaxes(pt, 1, 2) - p).max() < 1e-14
    assert abs(gt - g) <= 1e-12 * g


# ----------------------------------------------------- masks and structure
def test_mask_and_faces_invariant(oracle_mod):
    """Points with bnd = 0 (the faces and random interior points) never change
    and add nothing to the residual."""
    I, J, K = 10, 9, 12
    f = ji.himeno_fields(I, J, K, seed=9)
    rng = np.random.default_rng(1)
    holes = rng.random(f["bnd"].shape) < 0.2
    f["bnd"] = np.where(holes, 0.0, f["bnd"])
    p, g = oracle_mod.run(f, 6, OMEGA)
    frozen = f["bnd"] == 0.0
    assert np.array_equal(p[frozen], f["p"][frozen])
    # residual counts only bnd = 1 points: compare with the update it made
    p5, _ = oracle_mod.run(f, 5, OMEGA)
    ss = (p - p5) / OMEGA
    assert abs(g - np.sum(ss ** 2)) <= 1e-12 * g


def test_residual_is_taken_from_the_sweep_input(oracle_mod):
    """gosa of sweep n equals sum((p_n - p_{n-1}) / omega)^2, which uses the
    same ss as the update of sweep n (not of sweep n+1)."""
    f = ji.himeno_fields(9, 9, 9, seed=2)
    p3, _ = oracle_mod.run(f, 3, OMEGA)
    p4, g4 = oracle_mod.run(f, 4, OMEGA)
    assert abs(g4 - np.sum(((p4 - p3) / OMEGA) ** 2)) <= 1e-10 * g4


def test_jacobi_not_gauss_seidel(oracle_mod):
    """A Jacobi sweep is the same map whatever order the points are visited:
    sweeping the reversed grid (all three axes mirrored) gives the mirrored
    result, which an in-place update would not."""
    f = ji.himeno_fields(8, 7, 9, seed=6)
    p, _ = oracle_mod.run(f, 1, OMEGA)
    fr = mirror(mirror(mirror(f, 0), 1), 2)
    pr, _ = oracle_mod.run(fr, 1, OMEGA)
    assert np.abs(np.flip(pr, (0, 1, 2)) - p).max() < 1e-14
    # and each point depends only on the input state: change p at one point
    x = (4, 3, 4)
    q = f["p"].copy()
    q[x] += 1.0
    pq, _ = oracle_mod.sweep(f, q, OMEGA)
    p1, _ = oracle_mod.sweep(f, f["p"], OMEGA)
    changed = np.argwhere(np.abs(pq - p1) > 0)
    assert (np.abs(changed - np.array(x)).max(axis=1) <= 1).all()


def test_omega_zero_is_identity(oracle_mod):
    f = ji.himeno_fields(6, 6, 6, seed=8)
    p, g = oracle_mod.run(f, 3, 0.0)
    assert np.array_equal(p, f["p"]) and g > 0


def test_one_sweep_derivative_in_wrk1(oracle_mod):
    """A sweep is affine in wrk1 with slope omega * bnd * a3 at each point."""
    f = ji.himeno_fields(7, 7, 7, seed=12)
    rng = np.random.default_rng(3)
    d = rng.uniform(-1, 1, f["wrk1"].shape)
    p1, _ = oracle_mod.sweep(f, f["p"], OMEGA)
    g = dict(f)
    g["wrk1"] = f["wrk1"] + d
    p2, _ = oracle_mod.sweep(g, f["p"], OMEGA)
    assert np.abs((p2 - p1) - OMEGA * f["bnd"] * f["a3"] * d).max() < 1e-15


def test_superposition_over_sweeps(oracle_mod):
    """With wrk1 = 0 a sweep is linear in the state (faces included: they are
    copied), so n sweeps of a p1 + b p2 equal a (n sweeps of p1) + b (n
    sweeps of p2); and n sweeps are affine in wrk1, so the change that adding
    w2 to wrk1 makes does not depend on the wrk1 it is added to.  A term
    that is not linear in p (a constant, an |x|, a product of two states)
    breaks the first; a wrk1 weighted by the state breaks the second."""
    I, J, K, n = 8, 7, 9, 4
    f = ji.himeno_fields(I, J, K, seed=21)
    rng = np.random.default_rng(21)
    f0 = dict(f)
    f0["wrk1"] = np.zeros_like(f["wrk1"])
    p1, p2 = rng.uniform(-1, 1, f["p"].shape), rng.uniform(-1, 1, f["p"].shape)
    a, b = 0.7, -1.3
    q1, _ = oracle_mod.run(f0, n, OMEGA, p0=p1)
    q2, _ = oracle_mod.run(f0, n, OMEGA, p0=p2)
    q12, _ = oracle_mod.run(f0, n, OMEGA, p0=a * p1 + b * p2)
    assert np.abs(q12 - (a * q1 + b * q2)).max() < 1e-13
    w1, w2 = rng.uniform(-1, 1, f["p"].shape), rng.uniform(-1, 1, f["p"].shape)

    def with_wrk1(w):
        g = dict(f)
        g["wrk1"] = w
        return oracle_mod.run(g, n, OMEGA)[0]

    d_at_w1 = with_wrk1(w1 + w2) - with_wrk1(w1)
    d_at_0 = with_wrk1(w2) - with_wrk1(np.zeros_like(w2))
    assert np.abs(d_at_w1 - d_at_0).max() < 1e-13
    assert np.abs(d_at_0).max() > 1e-2          # wrk1 does move the state


def _longhand_point(P, f, i, j, k):
    """One point's update written out term by term from the workload's
    definition of the stencil (arrays indexed [k, j, i])."""
    a0, a1, a2, a3 = f["a0"][k, j, i], f["a1"][k, j, i], f["a2"][k, j, i], f["a3"][k, j, i]
    b0, b1, b2 = f["b0"][k, j, i], f["b1"][k, j, i], f["b2"][k, j, i]
    c0, c1, c2 = f["c0"][k, j, i], f["c1"][k, j, i], f["c2"][k, j, i]
    s0 = (a0 * P[k, j, i + 1] + a1 * P[k, j + 1, i] + a2 * P[k + 1, j, i]
          + b0 * (P[k, j + 1, i + 1] - P[k, j - 1, i + 1] - P[k, j + 1, i - 1] + P[k, j - 1, i - 1])
          + b1 * (P[k + 1, j + 1, i] - P[k - 1, j + 1, i] - P[k + 1, j - 1, i] + P[k - 1, j - 1, i])
          + b2 * (P[k + 1, j, i + 1] - P[k - 1, j, i + 1] - P[k + 1, j, i - 1] + P[k - 1, j, i - 1])
          + c0 * P[k, j, i - 1] + c1 * P[k, j - 1, i] + c2 * P[k - 1, j, i]
          + f["wrk1"][k, j, i])
    ss = (s0 * a3 - P[k, j, i]) * f["bnd"][k, j, i]
    return P[k, j, i] + OMEGA * ss, ss


@pytest.mark.parametrize("n", [1, 2, 3])
def test_brute_force_4cubed_longhand(oracle_mod, n):
    """4^3 (eight interior points), one to three Jacobi sweeps: every point's
    19 terms written out by hand from the stencil's definition, each sweep
    reading only the previous state, the faces never written, and the
    residual the sum of the last sweep's ss^2.  One interior point is masked
    (bnd = 0).  Agreement to rounding of the same operations."""
    f = ji.himeno_fields(4, 4, 4, seed=41)
    f["bnd"] = f["bnd"].copy()
    f["bnd"][2, 1, 2] = 0.0
    P = f["p"].copy()
    for _ in range(n):
        new = P.copy()
        sq = []
        for k in (1, 2):
            for j in (1, 2):
                for i in (1, 2):
                    new[k, j, i], ss = _longhand_point(P, f, i, j, k)
                    sq.append(ss * ss)
        P = new
    gosa = float(np.sum(sq))
    got_p, got_g = oracle_mod.run(f, n, OMEGA)
    assert np.abs(got_p - P).max() <= 1e-15 * np.abs(P).max()
    assert abs(got_g - gosa) <= 1e-14 * gosa
    assert got_p[2, 1, 2] == f["p"][2, 1, 2]


def test_minimal_grid_single_point(oracle_mod):
    """3^3 has one interior point; its new value is an affine function of its
    18 neighbours with slopes a3*coef (sign of each b corner), checked by
    moving one neighbour at a time."""
    f = ji.himeno_fields(3, 3, 3, seed=21)
    base, _ = oracle_mod.sweep(f, f["p"], OMEGA)
    c = (1, 1, 1)
    a3 = f["a3"][c]
    want = {(1, 1, 2): f["a0"][c], (1, 1, 0): f["c0"][c], (1, 2, 1): f["a1"][c],
            (1, 0, 1): f["c1"][c], (2, 1, 1): f["a2"][c], (0, 1, 1): f["c2"][c]}
    for (dk, dj, di), s in (((1, 2, 2), 1), ((1, 0, 2), -1), ((1, 2, 0), -1), ((1, 0, 0), 1)):
        want[(dk, dj, di)] = s * f["b0"][c]
    for (dk, dj, di), s in (((2, 2, 1), 1), ((0, 2, 1), -1), ((2, 0, 1), -1), ((0, 0, 1), 1)):
        want[(dk, dj, di)] = s * f["b1"][c]
    for (dk, dj, di), s in (((2, 1, 2), 1), ((0, 1, 2), -1), ((2, 1, 0), -1), ((0, 1, 0), 1)):
        want[(dk, dj, di)] = s * f["b2"][c]
    assert len(want) == 18
    for pos in np.ndindex(3, 3, 3):
        q = f["p"].copy()
        q[pos] += 1.0
        pq, _ = oracle_mod.sweep(f, q, OMEGA)
        slope = pq[c] - base[c]
        if pos == c:
            expect = 1.0 - OMEGA
        elif pos in want:
            expect = OMEGA * a3 * want[pos]
        else:
            expect = 0.0                    # the 8 cube corners are not read
        assert abs(slope - expect) < 1e-14, pos


def test_state_f32_rounds_new_values(oracle_mod):
    f = oracle_mod.round_inputs(ji.himeno_fields(6, 7, 8), "f32")
    p, _ = oracle_mod.run(f, 2, OMEGA, state="f32")
    assert np.array_equal(p, p.astype(np.float32).astype(np.float64))
    q, _ = oracle_mod.run(f, 2, OMEGA)
    assert 0 < np.abs(p - q).max() < 1e-6


def test_round_inputs_bf16_rule(oracle_mod):
    x = np.array([1.0, 1.00390625, 1.005859375, 1.0 + 2 ** -9 + 2 ** -24, -0.019])
    r = oracle_mod.bf16_round(x)
    # bf16 keeps 7 fraction bits: 1 + 2^-8 is a tie, rounded to even
    assert r[0] == 1.0
    assert r[1] == 1.0                 # 1 + 2^-8 ties to even (1.0)
    assert r[2] == 1.0078125           # 1 + 1.5*2^-8 rounds up
    assert r[3] == 1.0
    assert abs(r[4] + 0.019) < 2 ** -7 * 0.019
    f = ji.himeno_fields(4, 4, 4)
    rb = oracle_mod.round_inputs(f, "bf16")
    assert np.array_equal(rb["p"], f["p"].astype(np.float32).astype(np.float64))
    assert np.array_equal(rb["a0"], oracle_mod.bf16_round(f["a0"].astype(np.float32)))


# ------------------------------------------------------------------ adjoint
def _loss(p, target):
    d = p - target
    return 0.5 * np.sum(d * d)


def test_adjoint_matches_central_differences(oracle_mod):
    """Gradients of L = 1/2 |p_T - target|^2 against central differences of
    the forward oracle.  L is quadratic in wrk1 (the sweeps are affine in it),
    so the wrk1 check is exact up to rounding; a3 and the other coefficients
    enter polynomially.  h = 1e-6; the bar allows the rounding error of a
    central difference, about eps * L / h, on top of 1e-6 max|g| + 1e-5 |g|.
    L is quadratic in p0 as well (the sweeps are affine in the state), so
    that check is exact up to rounding too."""
    I, J, K, T = 9, 10, 11, 6
    f = ji.himeno_fields(I, J, K, seed=30)
    target = ji.target_field(I, J, K)
    adj = oracle_mod.adjoint(f, T, target, OMEGA, coef_grads=True)
    pT, _ = oracle_mod.run(f, T, OMEGA)
    assert np.array_equal(adj["pT"], pT)
    assert abs(adj["loss"] - _loss(pT, target)) <= 1e-14 * adj["loss"]
    pw, pa = ji.fd_points(I, J, K, 8)
    h = 1e-6
    gmax = {}
    # every parameter the adjoint differentiates: wrk1, a3, the nine stencil
    # coefficients and the initial state p0 (faces of p0 included: they are
    # read by the first sweep)
    names = ("wrk1", "a3", "a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2", "p")
    for q, name in enumerate(names):
        g = adj["g_p0" if name == "p" else "g_" + name]
        pts = (pw, pa)[q % 2]
        if name == "p":
            pts = list(pts) + [(0, 4, 5), (3, 0, 2), (I - 1, 5, 7)]
        for (i, j, k) in pts:
            fp = {n: v.copy() for n, v in f.items()}
            fm = {n: v.copy() for n, v in f.items()}
            fp[name][k, j, i] += h
            fm[name][k, j, i] -= h
            lp = _loss(oracle_mod.run(fp, T, OMEGA)[0], target)
            lm = _loss(oracle_mod.run(fm, T, OMEGA)[0], target)
            fd = (lp - lm) / (2 * h)
            # rounding of the two losses, divided by 2h, plus the O(h^2) term
            tol = 16 * np.finfo(float).eps * adj["loss"] / h + 1e-6 * np.abs(g).max() + 1e-5 * abs(fd)
            assert abs(fd - g[k, j, i]) <= tol, (name, i, j, k, fd, g[k, j, i])
    # faces carry no parameter gradient; the bnd = 0 centre has none either
    assert np.all(adj["g_wrk1"][0] == 0) and np.all(adj["g_a3"][:, :, -1] == 0)


def test_adjoint_dot_product_identity(oracle_mod):
    """<J d, lambda_T> = <d, J^T lambda_T> for directions d in (p0, wrk1); the
    map (p0, wrk1) -> p_T is affine, so J d = (p_T(+d) - p_T(-d)) / 2 exactly
    up to rounding."""
    I, J, K, T = 8, 9, 10, 7
    f = ji.himeno_fields(I, J, K, seed=31)
    target = ji.target_field(I, J, K)
    adj = oracle_mod.adjoint(f, T, target, OMEGA)
    lam = adj["pT"] - target
    rng = np.random.default_rng(7)
    dp = rng.uniform(-1, 1, f["p"].shape)
    dw = rng.uniform(-1, 1, f["p"].shape)
    fp = dict(f); fp["wrk1"] = f["wrk1"] + dw
    fm = dict(f); fm["wrk1"] = f["wrk1"] - dw
    pp, _ = oracle_mod.run(fp, T, OMEGA, p0=f["p"] + dp)
    pm, _ = oracle_mod.run(fm, T, OMEGA, p0=f["p"] - dp)
    lhs = np.sum(0.5 * (pp - pm) * lam)
    rhs = np.sum(dp * adj["g_p0"]) + np.sum(dw * adj["g_wrk1"])
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sum(np.abs(dp * adj["g_p0"])))


@pytest.mark.parametrize("state", ["f64", "f32"])
def test_sampled_points_equal_the_full_run(oracle_mod, state):
    """sample_after (each point from the oracle on the sub-box of radius n
    around it, the form the full-size GPU tests use) gives, bitwise, the full
    run's value: after n sweeps a point depends only on points within
    Chebyshev distance n, and the sub-box's held faces reach the centre only
    at sweep n + 1.  Points near the grid faces clip the box to the grid."""
    I, J, K, n = 21, 17, 15, 4
    f = ji.himeno_fields(I, J, K, seed=31)
    if state == "f32":
        f = oracle_mod.round_inputs(f, "f32")
    full, _ = oracle_mod.run(f, n, OMEGA, state=state)
    pts = [(10, 8, 7), (1, 1, 1), (I - 2, J - 2, K - 2), (5, 12, 2), (15, 3, 11)]
    got = oracle_mod.sample_after(f, n, pts, OMEGA, state=state)
    want = np.array([full[k, j, i] for i, j, k in pts])
    assert np.array_equal(got, want)
    # the radius is tight: a box of radius n - 1 holds faces that reach the
    # centre within n sweeps, and the value differs
    i, j, k = pts[0]
    r = n - 1
    sub = {name: np.ascontiguousarray(v[k - r:k + r + 1, j - r:j + r + 1, i - r:i + r + 1])
           for name, v in f.items()}
    p_small, _ = oracle_mod.run(sub, n, OMEGA, state=state)
    assert p_small[r, r, r] != full[k, j, i]
