"""Pins of the dense oracle against facts the paper and the mathematics fix:
planted factors, X.P(X^{-1}) = n, finite differences, special cases with
closed forms, Legendre/completion identities and exact rational brute force."""
import numpy as np
import pytest

from oracle import dense as OD
from oracle import symbolic as OS
import workloads as W


def filled(pattern):
    """Filled (chordal) pattern of a pattern in its given order, as lower CSC."""
    n, cp, ri = pattern
    I, _ = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    rows = np.concatenate([I[k] for k in range(n)]) if n else np.zeros(0, np.int64)
    cols = np.concatenate([np.full(len(I[k]), k) for k in range(n)])
    return W.lower_csc_from_pairs(n, rows, cols)


def random_chordal(seed, n=None, p=None):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(4, 25))
    p = p if p is not None else rng.uniform(0.05, 0.3)
    rows, cols = [], []
    for j in range(n):
        for i in range(j + 1, n):
            if rng.random() < p:
                rows.append(i)
                cols.append(j)
    return filled(W.lower_csc_from_pairs(n, np.array(rows, np.int64), np.array(cols, np.int64)))


PATTERNS = {
    "band": lambda: W.band(30, 4),
    "arrow": lambda: W.arrow(25, 4),
    "grid": lambda: filled(W.permute(W.grid2d(5, 5), W.nested_dissection((5, 5), leaf=4))),
    "random": lambda: random_chordal(3),
}


def spd_values(p, seed):
    n, cp, ri = p
    return W.diag_dominant(n, cp, ri, np.random.default_rng(seed))


# ---------------------------------------------------------------------------
# factor / logdet
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PATTERNS))
def test_factor_recovers_planted(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    x, l0, d0 = W.planted_factor(n, cp, ri, np.random.default_rng(5), dmin=1e-3)
    lv, d, outside = OD.factor(n, cp, ri, x)
    assert outside < 1e-12  # the factor of a filled pattern stays on V (Eq. (e-filled))
    np.testing.assert_allclose(d, d0, rtol=1e-9)
    np.testing.assert_allclose(lv, l0, rtol=0, atol=1e-9)
    assert abs(OD.logdet(n, cp, ri, x) - np.sum(np.log(d0))) < 1e-9 * max(1.0, abs(np.sum(np.log(d0))))


def test_factor_planted_cond_1e6():
    p = W.band(60, 6)
    n, cp, ri = p
    x, l0, d0 = W.planted_factor(n, cp, ri, np.random.default_rng(7), dmin=1e-6, dmax=1.0)
    lv, d, _ = OD.factor(n, cp, ri, x)
    np.testing.assert_allclose(d, d0, rtol=1e-6)
    np.testing.assert_allclose(lv, l0, rtol=0, atol=1e-6)


def test_factor_reconstructs_x():
    p = PATTERNS["grid"]()
    n, cp, ri = p
    x = spd_values(p, 1)
    lv, d, _ = OD.factor(n, cp, ri, x)
    r, c = OD.pattern_pairs(n, cp, ri)
    L = np.zeros((n, n))
    L[r, c] = lv
    X = L @ np.diag(d) @ L.T
    np.testing.assert_allclose(OD.project(n, cp, ri, X), x, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.diag(L), 1.0)


# ---------------------------------------------------------------------------
# gradient (Eq. (e-grad-def))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PATTERNS))
def test_trace_identity(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    x = spd_values(p, 2)
    s = OD.projected_inverse(n, cp, ri, x)
    # X.P(X^{-1}) = tr(X X^{-1}) = n since X is supported on V
    assert abs(OD.sym_dot(n, cp, ri, x, s) - n) < 1e-10 * n


@pytest.mark.parametrize("name", list(PATTERNS))
def test_gradient_finite_difference(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    x = spd_values(p, 3)
    y = W.uniform_sym(n, cp, ri, np.random.default_rng(4))[0]
    g = OD.gradient(n, cp, ri, x)
    h = 1e-5
    f = lambda v: -OD.logdet(n, cp, ri, v)
    fd = (f(x + h * y) - f(x - h * y)) / (2 * h)
    assert abs(fd - OD.sym_dot(n, cp, ri, g, y)) < 1e-6 * max(1.0, abs(fd))


def test_gradient_block_diagonal_closed_form():
    # X block diagonal with 2x2 blocks [[a, b], [b, c]]: inverse [[c, -b], [-b, a]] / (ac - b^2)
    n = 10
    rows = np.arange(1, n, 2)
    cols = np.arange(0, n, 2)
    n, cp, ri = W.lower_csc_from_pairs(n, rows, cols)
    rng = np.random.default_rng(0)
    x = np.zeros(len(ri))
    want = np.zeros(len(ri))
    for j in range(0, n, 2):
        a, b, c = rng.uniform(2, 3), rng.uniform(-1, 1), rng.uniform(2, 3)
        det = a * c - b * b
        x[cp[j]] = a; x[cp[j] + 1] = b; x[cp[j + 1]] = c
        want[cp[j]] = c / det; want[cp[j] + 1] = -b / det; want[cp[j + 1]] = a / det
    np.testing.assert_allclose(OD.gradient(n, cp, ri, x), -want, rtol=1e-13)


def test_gradient_diagonal_pattern():
    n = 12
    n, cp, ri = W.lower_csc_from_pairs(n, np.zeros(0, np.int64), np.zeros(0, np.int64))
    x = np.random.default_rng(1).uniform(0.5, 3, size=n)
    np.testing.assert_allclose(OD.gradient(n, cp, ri, x), -1.0 / x, rtol=1e-14)


# ---------------------------------------------------------------------------
# Hessian (§1.1, §5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PATTERNS))
def test_hessian_finite_difference_of_gradient(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    x = spd_values(p, 5)
    y = W.uniform_sym(n, cp, ri, np.random.default_rng(6))[0]
    t = OD.hessian(n, cp, ri, x, [y])[0]
    h = 1e-5
    fd = (OD.gradient(n, cp, ri, x + h * y) - OD.gradient(n, cp, ri, x - h * y)) / (2 * h)
    assert OD.rel_err(n, cp, ri, fd, t) < 1e-7


def test_hessian_identity_and_diagonal_x():
    p = PATTERNS["band"]()
    n, cp, ri = p
    r, c = OD.pattern_pairs(n, cp, ri)
    y = W.uniform_sym(n, cp, ri, np.random.default_rng(1))[0]
    eye = np.where(r == c, 1.0, 0.0)
    np.testing.assert_allclose(OD.hessian(n, cp, ri, eye, [y])[0], y, rtol=1e-14, atol=1e-15)
    dx = np.random.default_rng(2).uniform(0.5, 2.0, size=n)
    xd = np.where(r == c, dx[r], 0.0)
    want = y / (dx[r] * dx[c])
    np.testing.assert_allclose(OD.hessian(n, cp, ri, xd, [y])[0], want, rtol=1e-13)


@pytest.mark.parametrize("name", list(PATTERNS))
def test_hessian_self_adjoint_positive(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    x = spd_values(p, 8)
    y1, y2 = W.uniform_sym(n, cp, ri, np.random.default_rng(9), count=2)
    t1, t2 = OD.hessian(n, cp, ri, x, [y1, y2])
    a = OD.sym_dot(n, cp, ri, y1, t2)
    b = OD.sym_dot(n, cp, ri, y2, t1)
    assert abs(a - b) < 1e-12 * max(abs(a), 1.0)
    assert OD.sym_dot(n, cp, ri, y1, t1) > 0


@pytest.mark.parametrize("name", list(PATTERNS))
def test_hessian_entries(name):
    """Entries of X^{-1} Y X^{-1} one by one: X diagonal gives
    Y_ij / (x_i x_j) (closed form), a central difference of the gradient
    -P(X^{-1}) along Y gives H(Y) at the same positions, and the entries
    agree with the whole projected product."""
    p = PATTERNS[name]()
    n, cp, ri = p
    r, c = OD.pattern_pairs(n, cp, ri)
    rng = np.random.default_rng(21)
    y = W.uniform_sym(n, cp, ri, rng)[0]
    sel = rng.choice(len(r), size=min(40, len(r)), replace=False)
    dx = rng.uniform(0.5, 2.0, size=n)
    xd = np.where(r == c, dx[r], 0.0)
    Zd = OD.inverse(n, cp, ri, xd)
    got = OD.hessian_entries(n, cp, ri, Zd, y, r[sel], c[sel])
    np.testing.assert_allclose(got, y[sel] / (dx[r[sel]] * dx[c[sel]]), rtol=1e-13)
    x = spd_values(p, 22)
    Z = OD.inverse(n, cp, ri, x)
    got = OD.hessian_entries(n, cp, ri, Z, y, r[sel], c[sel])
    h = 1e-5
    fd = (OD.gradient(n, cp, ri, x + h * y) - OD.gradient(n, cp, ri, x - h * y)) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(got - fd[sel]).max() < 1e-7 * scale
    np.testing.assert_allclose(got, OD.hessian(n, cp, ri, x, [y], Z=Z)[0][sel], rtol=1e-11, atol=1e-14 * scale)


def test_hessian_matrix_consistent():
    p = PATTERNS["grid"]()
    n, cp, ri = p
    x = spd_values(p, 10)
    y = W.uniform_sym(n, cp, ri, np.random.default_rng(11))[0]
    Hm = OD.hessian_matrix(n, cp, ri, x)
    np.testing.assert_allclose(Hm @ y, OD.hessian(n, cp, ri, x, [y])[0], rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------------------
# inverse Hessian (§5.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PATTERNS))
def test_inverse_hessian_roundtrip_and_routes(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    x = spd_values(p, 12)
    t = W.uniform_sym(n, cp, ri, np.random.default_rng(13))[0]
    y_dense = OD.inv_hessian_dense(n, cp, ri, x, [t])[0]
    assert OD.rel_err(n, cp, ri, OD.hessian(n, cp, ri, x, [y_dense])[0], t) < 1e-11
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    y_cs = OD.inv_hessian_cliquesum(n, cp, ri, x, t, cl, seps)
    assert OD.rel_err(n, cp, ri, y_cs, y_dense) < 1e-10
    y_cg = OD.inv_hessian_cg(n, cp, ri, x, t)
    assert OD.rel_err(n, cp, ri, y_cg, y_dense) < 1e-9


def test_inverse_hessian_at_identity():
    p = PATTERNS["arrow"]()
    n, cp, ri = p
    r, c = OD.pattern_pairs(n, cp, ri)
    t = W.uniform_sym(n, cp, ri, np.random.default_rng(1))[0]
    eye = np.where(r == c, 1.0, 0.0)
    np.testing.assert_allclose(OD.inv_hessian_dense(n, cp, ri, eye, [t])[0], t, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# completion / dual barrier (§1.2, Eq. (e-Xhat-eq), (e-legendre-rels))
# ---------------------------------------------------------------------------

def gram_values(p, seed, k=5, c=0.5):
    n, cp, ri = p
    G = np.random.default_rng(seed).standard_normal((n, k))
    return W.projected_gram(n, cp, ri, G, c)


@pytest.mark.parametrize("name", list(PATTERNS))
def test_completion_newton_vs_cliquesum(name):
    p = PATTERNS[name]()
    n, cp, ri = p
    s = gram_values(p, 14)
    xn = OD.completion_newton(n, cp, ri, s)
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    xc = OD.completion_cliquesum(n, cp, ri, s, cl, seps)
    # P(Xhat^{-1}) = S (Eq. (e-Xhat-eq)) for both
    for xh in (xn, xc):
        assert OD.rel_err(n, cp, ri, OD.projected_inverse(n, cp, ri, xh), s) < 1e-12
    assert OD.rel_err(n, cp, ri, xn, xc) < 1e-11
    # S.Xhat = n and f_* = log det Xhat - n equals the sup value -S.Xhat + log det Xhat
    fstar = OD.dual_barrier(n, cp, ri, xc)
    assert abs(OD.sym_dot(n, cp, ri, s, xc) - n) < 1e-10 * n
    val = -OD.sym_dot(n, cp, ri, s, xc) + OD.logdet(n, cp, ri, xc)
    assert abs(val - fstar) < 1e-10 * max(1.0, abs(fstar))
    # the sup is attained at Xhat: nearby X in S_V do not do better
    rng = np.random.default_rng(15)
    for _ in range(5):
        d = W.uniform_sym(n, cp, ri, rng)[0]
        xp = xc + 1e-3 * d
        assert -OD.sym_dot(n, cp, ri, s, xp) + OD.logdet(n, cp, ri, xp) <= val + 1e-12


@pytest.mark.parametrize("name", list(PATTERNS))
def test_completion_refined(name):
    """Newton steps from the closed form reach the maximiser of
    Eq. (e-dual-barrier-def) that Newton from diag(1/S_ii) reaches, and
    satisfy P(X^{-1}) = S (Eq. (e-Xhat-eq)) to rounding."""
    p = PATTERNS[name]()
    n, cp, ri = p
    s = gram_values(p, 15, c=0.01)
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    xr = OD.completion_refined(n, cp, ri, s, cl, seps)
    xn = OD.completion_newton(n, cp, ri, s)
    assert OD.rel_err(n, cp, ri, xr, xn) < 1e-11
    Z = np.linalg.inv(OD.to_dense(n, cp, ri, xr))
    assert OD.rel_err(n, cp, ri, OD.project(n, cp, ri, Z), s) < 1e-13


def test_completion_refined_removes_closed_form_residual():
    """On a larger, ill-conditioned S (an Erdos-Renyi pattern under minimum
    fill, S = P(G G^T + 0.01 I), cond(X-hat) about 1e5) the closed form's
    residual ||P(X^{-1}) - S|| / ||S|| (about 3e-8) is brought to the
    rounding floor of P(X^{-1}) by the Newton steps."""
    rng = np.random.default_rng(16)
    p = filled(W.erdos_renyi(400, 0.01, rng))
    n, cp, ri = p
    s = W.projected_gram(n, cp, ri, rng.standard_normal((n, 30)), 1e-2)
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    res = lambda xv: OD.rel_err(n, cp, ri, OD.project(n, cp, ri, np.linalg.inv(OD.to_dense(n, cp, ri, xv))), s)
    r0 = res(OD.completion_cliquesum(n, cp, ri, s, cl, seps))
    r1 = res(OD.completion_refined(n, cp, ri, s, cl, seps))
    assert r1 < 1e-3 * r0 and r1 < 1e-11


def test_completion_tridiagonal_by_hand():
    # band 1: cliques {k, k+1}, separators {k}; Xhat = sum_k E [[a b][b c]]^{-1} E^T - sum e_k e_k^T / s_kk
    n = 9
    p = W.band(n, 1)
    n, cp, ri = p
    s = gram_values(p, 16, k=3, c=1.0)
    S = OD.to_dense(n, cp, ri, s)
    Xh = np.zeros((n, n))
    for k in range(n - 1):
        a, b, c = S[k, k], S[k + 1, k], S[k + 1, k + 1]
        det = a * c - b * b
        Xh[k, k] += c / det; Xh[k + 1, k + 1] += a / det
        Xh[k + 1, k] += -b / det; Xh[k, k + 1] += -b / det
    for k in range(1, n - 1):
        Xh[k, k] -= 1.0 / S[k, k]
    want = OD.project(n, cp, ri, Xh)
    np.testing.assert_allclose(OD.completion_newton(n, cp, ri, s), want, rtol=1e-11)


def test_completion_special_patterns():
    rng = np.random.default_rng(17)
    # diagonal pattern: Xhat = diag(1/S_ii)
    n = 7
    n, cp, ri = W.lower_csc_from_pairs(n, np.zeros(0, np.int64), np.zeros(0, np.int64))
    s = rng.uniform(0.5, 2.0, size=n)
    np.testing.assert_allclose(OD.completion_newton(n, cp, ri, s), 1.0 / s, rtol=1e-13)
    # full pattern: P(Xhat^{-1}) = S means Xhat = S^{-1}; S^{-1} checked by S Xhat = I
    p = W.band(6, 5)
    n, cp, ri = p
    s = gram_values(p, 18, k=6, c=0.5)
    xh = OD.completion_newton(n, cp, ri, s)
    np.testing.assert_allclose(OD.to_dense(n, cp, ri, s) @ OD.to_dense(n, cp, ri, xh), np.eye(n),
                               atol=1e-12)


def test_legendre_inverse_hessian_at_xhat():
    # grad^2 f_*(S) = grad^2 f(Xhat)^{-1} (Eq. (e-legendre-rels)): the derivative of
    # S -> Xhat(S) along T equals -H_{Xhat}^{-1}(T)
    p = PATTERNS["grid"]()
    n, cp, ri = p
    s = gram_values(p, 19)
    t = W.uniform_sym(n, cp, ri, np.random.default_rng(20))[0]
    I, parent = OS.fill(n, OS.columns_from_csc(n, cp, ri))
    cl, seps = OS.cliques_and_separators(I, parent)
    xh = OD.completion_cliquesum(n, cp, ri, s, cl, seps)
    h = 1e-6
    d = (OD.completion_cliquesum(n, cp, ri, s + h * t, cl, seps)
         - OD.completion_cliquesum(n, cp, ri, s - h * t, cl, seps)) / (2 * h)
    want = -OD.inv_hessian_dense(n, cp, ri, xh, [t])[0]
    assert OD.rel_err(n, cp, ri, d, want) < 1e-7


# ---------------------------------------------------------------------------
# exact rational brute force on tiny chordal patterns
# ---------------------------------------------------------------------------

def _exact_case(seed):
    sp = pytest.importorskip("sympy")
    p = random_chordal(seed, n=5, p=0.45)
    n, cp, ri = p
    rng = np.random.default_rng(seed)
    r, c = OD.pattern_pairs(n, cp, ri)
    # small integers: X diagonally dominant, Y arbitrary
    xi = np.where(r == c, 0, rng.integers(-3, 4, size=len(r)))
    rows = np.zeros(n, dtype=np.int64)
    np.add.at(rows, r[r != c], np.abs(xi[r != c]))
    np.add.at(rows, c[r != c], np.abs(xi[r != c]))
    xi = np.where(r == c, rows[r] + 2, xi)
    yi = rng.integers(-3, 4, size=len(r))
    X = sp.zeros(n, n)
    Y = sp.zeros(n, n)
    for k in range(len(r)):
        X[int(r[k]), int(c[k])] = X[int(c[k]), int(r[k])] = int(xi[k])
        Y[int(r[k]), int(c[k])] = Y[int(c[k]), int(r[k])] = int(yi[k])
    return sp, p, r, c, X, Y, xi.astype(float), yi.astype(float)


@pytest.mark.parametrize("seed", range(6))
def test_exact_rational_gradient_hessian(seed):
    sp, p, r, c, X, Y, x, y = _exact_case(seed)
    n, cp, ri = p
    Z = X.inv()
    ZYZ = Z * Y * Z
    g_exact = np.array([-float(Z[int(a), int(b)]) for a, b in zip(r, c)])
    t_exact = np.array([float(ZYZ[int(a), int(b)]) for a, b in zip(r, c)])
    ld_exact = float(sp.log(X.det()))
    np.testing.assert_allclose(OD.gradient(n, cp, ri, x), g_exact, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(OD.hessian(n, cp, ri, x, [y])[0], t_exact, rtol=1e-12, atol=1e-14)
    assert abs(OD.logdet(n, cp, ri, x) - ld_exact) < 1e-13 * max(1, abs(ld_exact))


@pytest.mark.parametrize("seed", range(6))
def test_exact_rational_inverse_hessian_and_completion(seed):
    sp, p, r, c, X, Y, x, y = _exact_case(seed)
    n, cp, ri = p
    Z = X.inv()
    # exact H^{-1}(T) for T = H(Y) is Y itself; solve the exact linear system for T = Y too
    m = len(r)
    syms = sp.symbols(f"u0:{m}")
    U = sp.zeros(n, n)
    for k in range(m):
        U[int(r[k]), int(c[k])] = syms[k]
        U[int(c[k]), int(r[k])] = syms[k]
    HU = Z * U * Z
    eqs = [sp.Eq(HU[int(a), int(b)], int(y[k])) for k, (a, b) in enumerate(zip(r, c))]
    sol = sp.solve(eqs, syms, dict=True)[0]
    u_exact = np.array([float(sol[s]) for s in syms])
    np.testing.assert_allclose(OD.inv_hessian_dense(n, cp, ri, x, [y])[0], u_exact, rtol=1e-11, atol=1e-12)
    # completion of S = P(X^{-1}) is X itself (Eq. (e-Xhat-eq) has the unique solution X)
    s = np.array([float(Z[int(a), int(b)]) for a, b in zip(r, c)])
    np.testing.assert_allclose(OD.completion_newton(n, cp, ri, s), x, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------------------
# linearized factorization and Hessian factor (§5.1, §5.4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PATTERNS))
def test_linearized_factor_is_the_derivative(name):
    """L', D' against central differences of the dense LDL^T factor."""
    p = PATTERNS[name]()
    n, cp, ri = p
    rng = np.random.default_rng(91)
    x = spd_values(p, 92)
    y = W.uniform_sym(n, cp, ri, rng, count=1)[0]
    Lp, dp, L, d = OD.linearized_factor(n, cp, ri, x, y)
    h = 1e-5

    def ldl(v):
        C = np.linalg.cholesky(OD.to_dense(n, cp, ri, v))
        return C / np.diag(C)[None, :], np.diag(C) ** 2

    (La, da), (Lb, db) = ldl(x + h * y), ldl(x - h * y)
    np.testing.assert_allclose(dp, (da - db) / (2 * h), rtol=0, atol=1e-7 * np.max(np.abs(dp)))
    np.testing.assert_allclose(Lp, (La - Lb) / (2 * h), rtol=0, atol=1e-7 * max(1.0, np.max(np.abs(Lp))))
    # L' lives on the strictly lower part of the filled pattern
    mask = np.zeros((n, n), bool)
    rr, cc = OD.pattern_pairs(n, cp, ri)
    mask[rr, cc] = True
    assert np.max(np.abs(Lp[~mask | np.eye(n, dtype=bool)]), initial=0.0) < 1e-12 * max(1.0, np.max(np.abs(Lp)))


def test_reverse_cholesky_is_upper_factor():
    rng = np.random.default_rng(93)
    B = rng.standard_normal((7, 7))
    A = B @ B.T + 7 * np.eye(7)
    R = OD.reverse_cholesky(A)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(R @ R.T, A, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("name", list(PATTERNS))
def test_hessian_factor_composes_to_hessian(name):
    """H = R^adj o R (§5.4) against the dense definition of H, and R^adj is
    the adjoint of R in the trace inner product."""
    p = PATTERNS[name]()
    n, cp, ri = p
    rng = np.random.default_rng(94)
    x = spd_values(p, 95)
    ys = W.uniform_sym(n, cp, ri, rng, count=2)
    parts = OD.hessian_factor_parts(n, cp, ri, x)
    for I, R in parts:  # the factor the paper prescribes: upper, S_II = R R^T
        assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    w = OD.hessian_factor(n, cp, ri, x, list(ys), parts=parts)
    t = OD.hessian_factor_adj(n, cp, ri, x, w, parts=parts)
    h = OD.hessian(n, cp, ri, x, list(ys))
    for j in range(2):
        assert OD.rel_err(n, cp, ri, t[j], h[j]) < 1e-11
    # <R(Y0), W1> = <Y0, R^adj(W1)> for an unrelated W1
    w1 = W.uniform_sym(n, cp, ri, rng, count=1)[0]
    lhs = OD.sym_dot(n, cp, ri, w[0], w1)
    rhs = OD.sym_dot(n, cp, ri, ys[0], OD.hessian_factor_adj(n, cp, ri, x, [w1], parts=parts)[0])
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))
    # <Y, H(Y)> = ||R(Y)||^2
    assert abs(OD.sym_dot(n, cp, ri, ys[0], h[0]) - OD.sym_dot(n, cp, ri, w[0], w[0])) < 1e-10 * abs(
        OD.sym_dot(n, cp, ri, ys[0], h[0]))


def test_hessian_factor_diagonal_x_closed_form():
    """X diagonal: L = I, D = diag(x), S = diag(1/x), so R_j = diag(1/sqrt(x_I))
    and W_ij = Y_ij / sqrt(x_i x_j)."""
    n, cp, ri = W.band(12, 3)
    rng = np.random.default_rng(96)
    rr, cc = OD.pattern_pairs(n, cp, ri)
    xd = rng.uniform(0.5, 2.0, n)
    x = np.where(rr == cc, xd[rr], 0.0)
    y = W.uniform_sym(n, cp, ri, rng, count=1)[0]
    w = OD.hessian_factor(n, cp, ri, x, [y])[0]
    np.testing.assert_allclose(w, y / np.sqrt(xd[rr] * xd[cc]), rtol=1e-13, atol=0)


def test_hessian_factor_dense_2x2_by_hand():
    """Dense 2 x 2 pattern: X = [[a, b], [b, c]], D_11 = a, L_21 = b/a,
    D_22 = c - b^2/a.  For Y = E_21 + E_12: D'_11 = 0, L'_21 = 1/a,
    D'_22 = -2b/a; S_22 = 1/D_22 gives R_1 = 1/sqrt(D_22).  So
    W_11 = 0, W_21 = sqrt(a) (1/a) / sqrt(D_22), W_22 = D'_22 / D_22."""
    n, cp, ri = 2, np.array([0, 2, 3], np.int64), np.array([0, 1, 1], np.int32)
    a, b, c = 3.0, 1.0, 2.0
    x = np.array([a, b, c])
    y = np.array([0.0, 1.0, 0.0])
    d22 = c - b * b / a
    w = OD.hessian_factor(n, cp, ri, x, [y])[0]
    np.testing.assert_allclose(w, [0.0, np.sqrt(a) / a / np.sqrt(d22), (-2 * b / a) / d22], rtol=1e-14, atol=1e-15)


def fig_spy_w():
    """Figure 1's pattern and the W = R(Y) sparsity of Figure fig-spy-W."""
    import os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    pairs = np.loadtxt(os.path.join(gold, "fig1_pattern.txt"), dtype=np.int64, comments="#")
    pattern = W.lower_csc_from_pairs(17, pairs[:, 0], pairs[:, 1])
    cases, cur = {}, None
    with open(os.path.join(gold, "fig_spy_W.txt")) as f:
        for line in f:
            tok = line.split("#")[0].split()
            if not tok:
                continue
            if tok[0] == "case":
                cur = cases.setdefault(tok[1], {"y": None, "w": set()})
            elif tok[0] == "y":
                cur["y"] = (int(tok[1]), int(tok[2]))
            else:
                cur["w"].add((int(tok[1]), int(tok[2])))
    return pattern, cases


def spy(n, cp, ri, w, rel=1e-12):
    rr, cc = OD.pattern_pairs(n, cp, ri)
    big = np.abs(w) > rel * np.abs(w).max()
    return {(int(r), int(c)) for r, c, b in zip(rr, cc, big) if b}


@pytest.mark.parametrize("case", ["a", "b"])
def test_hessian_factor_sparsity_of_figure(case):
    """Figure fig-spy-W (§5.5): nonzeros of R(Y) for a Y with one nonzero; in
    case b the zero at (2, 1) next to the nonzero at (3, 1) holds only for
    the upper triangular R_j of Algorithm 5.3."""
    (n, cp, ri), cases = fig_spy_w()
    x = W.diag_dominant(n, cp, ri, np.random.default_rng(97))
    rr, cc = OD.pattern_pairs(n, cp, ri)
    y = np.where((rr == cases[case]["y"][0]) & (cc == cases[case]["y"][1]), 1.0, 0.0)
    w = OD.hessian_factor(n, cp, ri, x, [y])[0]
    assert spy(n, cp, ri, w) == cases[case]["w"]
