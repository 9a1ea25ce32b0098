"""Pins for the oracle's extensions of the interpolation, named by the paper
as directions it did not take (Section 6): piecewise quadratic Lagrange and
cubic Hermite bases in the wave speed, and bivariate interpolation in (c, a)
for damping that does not follow the wave speed.  Each pin is fixed by
mathematics, not by re-running the oracle: polynomial reproduction, the
order of convergence, linearity against the direct O(n^2) sum, and
exactness at node values.  None of these tests needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def _nodes_on_unit_range(M, basis, omega=30.0):
    med = O.make_medium(np.array([[1.0, 2.0], [1.5, 1.2]]), None, None, omega, M=M, c_o=1.0,
                        alpha=0.0, a_node=6.0, basis=basis)
    return med.nodes


# --------------------------------------------------------------------------
# Quadratic Lagrange basis in c
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M", [3, 5, 9])
def test_lagrange_basis_reproduces_quadratics(M):
    """Lagrange polynomials of degree 2 on each element reproduce 1, c and c^2
    exactly; at most three weights per point are non-zero and some are
    negative.  The hats of Eqn. 405 reproduce 1 and c but not c^2."""
    nodes = _nodes_on_unit_range(M, 1)
    cs = np.linspace(1.0, 2.0, 257).reshape(-1, 1)
    W = O.hat_weights(cs, np.zeros_like(cs), nodes)[:, :, 0]
    ck = nodes.c_real.reshape(-1, 1)
    x = cs[:, 0]
    np.testing.assert_allclose(W.sum(0), 1.0, atol=1e-14)
    np.testing.assert_allclose((W * ck).sum(0), x, atol=1e-13)
    np.testing.assert_allclose((W * ck ** 2).sum(0), x ** 2, atol=1e-13)
    assert (np.count_nonzero(W, axis=0) <= 3).all()
    assert (W < -1e-3).any()
    lin = O.hat_weights(cs, np.zeros_like(cs), _nodes_on_unit_range(M, 0))[:, :, 0]
    assert np.abs((lin * ck ** 2).sum(0) - x ** 2).max() > 1e-3


def test_lagrange_nodes_keep_c_o_on_an_element_boundary():
    """With c_o strictly inside the range, both equispaced segments get an
    even number of intervals, so c_o is the end node of an element."""
    cr = O.real_nodes(0.8, 3.6, 13, 1.0, basis=1)
    assert len(cr) == 13
    i_o = int(np.nonzero(cr == 1.0)[0][0])
    assert i_o % 2 == 0 and i_o >= 2 and (12 - i_o) % 2 == 0
    np.testing.assert_allclose(np.diff(cr[:i_o + 1]), (1.0 - 0.8) / i_o)
    np.testing.assert_allclose(np.diff(cr[i_o:]), (3.6 - 1.0) / (12 - i_o))
    with pytest.raises(ValueError):
        O.real_nodes(1.0, 2.0, 6, None, basis=1)


def _smooth_speed(shape):
    X = S.coords(shape)
    return 1.0 + 0.5 * (1 + np.cos(2 * np.pi * X[1])) * (1 + np.cos(2 * np.pi * X[0])) / 4


def test_lagrange_interpolation_converges_third_order():
    """Degree-2 interpolation of the symbol in c: ||(Q - Q_M) v|| falls like
    h_M^3 (the hats of Thm. Acc give h_M^2); direct un-interpolated Q as the
    reference."""
    shape = (12, 12)
    c = _smooth_speed(shape)
    v = S.random_field(rng(8), shape)
    ref = None
    slopes = {}
    for basis in (0, 1):
        errs, hs = [], []
        for M in (5, 9, 17, 33):
            med = O.make_medium(c, None, None, 20.0, M=M, c_o=1.0, alpha=0.5, basis=basis)
            if ref is None:
                ref = O.apply_pdo_direct(O.exact_symbol_at_point(med), v)
            errs.append(np.linalg.norm(O.apply_preconditioner(med, v) - ref))
            hs.append((c.max() - c.min()) / (M - 1))
        slopes[basis] = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 1.7 < slopes[0] < 2.5, slopes
    assert 2.6 < slopes[1] < 3.5, slopes


# --------------------------------------------------------------------------
# Piecewise cubic Hermite basis in c (values and c-derivatives at the nodes)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M", [2, 4, 7])
def test_hermite_basis_reproduces_cubics(M):
    """With node values f(c_k) on the value planes and node derivatives
    f'(c_k) on the derivative planes, the cubic Hermite weights reproduce
    every cubic f exactly (and not c^4); at most four weights per point are
    non-zero, and the value weights alone sum to one."""
    nodes = _nodes_on_unit_range(M, 2)
    assert nodes.K == 2 * M and list(nodes.deriv) == [0] * M + [1] * M
    cs = np.linspace(1.0, 2.0, 301).reshape(-1, 1)
    W = O.hat_weights(cs, np.zeros_like(cs), nodes)[:, :, 0]
    ck = nodes.c_real
    x = cs[:, 0]
    Wv, Wd = W[:M], W[M:]
    np.testing.assert_allclose(Wv.sum(0), 1.0, atol=1e-14)
    for f, df in ((lambda c: 1 + 0 * c, lambda c: 0 * c), (lambda c: c, lambda c: 1 + 0 * c),
                  (lambda c: c ** 2, lambda c: 2 * c), (lambda c: c ** 3 - 2 * c, lambda c: 3 * c ** 2 - 2)):
        got = (Wv * f(ck)[:, None]).sum(0) + (Wd * df(ck)[:, None]).sum(0)
        np.testing.assert_allclose(got, f(x), atol=1e-12)
    got4 = (Wv * (ck ** 4)[:, None]).sum(0) + (Wd * (4 * ck ** 3)[:, None]).sum(0)
    assert np.abs(got4 - x ** 4).max() > 1e-5
    assert (np.count_nonzero(W, axis=0) <= 4).all()


def test_symbol_derivative_in_c():
    """node_symbol_dc is the derivative of node_symbol in the wave speed: a
    central difference of Eqn. 021's symbol agrees to O(step^2)."""
    xi2 = np.linspace(0.0, 4000.0, 41)
    for c, a in ((1.3, 6.0), (2.1, 0.5)):
        d = 1e-5
        fd = (O.node_symbol(c + d, a, 30.0, xi2) - O.node_symbol(c - d, a, 30.0, xi2)) / (2 * d)
        np.testing.assert_allclose(O.node_symbol_dc(c, a, 30.0, xi2), fd, rtol=1e-6, atol=1e-12)


def test_hermite_interpolation_converges_fourth_order():
    """Cubic Hermite interpolation of the symbol in c: ||(Q - Q_M) v|| falls
    like h_M^4 (hats: h_M^2); the direct un-interpolated Q is the reference."""
    shape = (12, 12)
    c = _smooth_speed(shape)
    v = S.random_field(rng(8), shape)
    med0 = O.make_medium(c, None, None, 20.0, M=3, c_o=1.0, alpha=0.5, basis=2)
    ref = O.apply_pdo_direct(O.exact_symbol_at_point(med0), v)
    errs, hs = [], []
    for M in (5, 9, 17, 33):
        med = O.make_medium(c, None, None, 20.0, M=M, c_o=1.0, alpha=0.5, basis=2)
        errs.append(np.linalg.norm(O.apply_preconditioner(med, v) - ref))
        hs.append((c.max() - c.min()) / (M - 1))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 3.5 < slope < 4.6, (slope, errs)


def test_hermite_fft_apply_equals_direct_sum_with_layer():
    """The K FFT form (value and derivative planes, hats in zeta in the
    layer) equals the direct O(n^2) Op(q_M) with the interpolated symbol, and
    is exact where c takes node values (the derivative weights vanish
    there)."""
    p = S.small_problem((12, 10), 5, M=4, Mt=2, width=2)
    med = O.make_medium(p.c, p.zeta, None, p.omega, 4, 2, 1.0, None, 0.2, basis=2)
    v = S.random_field(rng(3), p.shape)
    fft = O.apply_preconditioner(med, v)
    direct = O.apply_pdo_direct(O.interpolated_symbol_at_point(med), v)
    assert np.linalg.norm(fft - direct) <= 1e-12 * np.linalg.norm(direct)
    c = np.full((8, 8), 1.0)
    c[2:6, 2:6] = 2.0
    med = O.make_medium(c, None, None, 15.0, M=3, c_o=1.0, alpha=0.2, basis=2)
    v = S.random_field(rng(4), c.shape)
    exact = O.apply_pdo_direct(O.exact_symbol_at_point(med), v)
    assert np.linalg.norm(O.apply_preconditioner(med, v) - exact) <= 1e-12 * np.linalg.norm(exact)


# --------------------------------------------------------------------------
# Bivariate interpolation in (c, a)
# --------------------------------------------------------------------------

def _independent_damping(shape):
    X = S.coords(shape)
    return 2.0 + 10.0 * (1 + np.sin(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[1])) / 2


def test_bivariate_weights_reproduce_bilinear_functions():
    """Tensor products of hats reproduce every f = p + q c + r a + s c a:
    sum_k w_k(x) f(c_k, a_k) = f(c(x), a(x)); at most four weights per point
    are non-zero.  c^2 a is not reproduced (hats are linear in c)."""
    shape = (10, 8)
    c = _smooth_speed(shape)
    a = _independent_damping(shape)
    med = O.make_medium(c, None, a, 20.0, M=4, c_o=1.0, alpha=0.3, Ma=3)
    nd = med.nodes
    assert nd.K == 12 and nd.Ma == 3 and nd.Ks == 4
    ck = nd.gamma.real.reshape((-1,) + (1,) * c.ndim)
    ak = np.array([nd.a_nodes[k % nd.Ma] for k in range(nd.K)]).reshape(ck.shape)
    np.testing.assert_allclose(nd.a, ak.ravel() + 0.3 * 20.0, rtol=1e-15)
    W = med.W
    for f in (lambda cc, aa: 1.0 + 0 * cc, lambda cc, aa: cc, lambda cc, aa: aa,
              lambda cc, aa: 3.0 - 2.0 * cc + 0.5 * aa + 1.5 * cc * aa):
        np.testing.assert_allclose((W * f(ck, ak)).sum(0), f(c, a), atol=1e-12)
    assert (np.count_nonzero(W.reshape(nd.K, -1), axis=0) <= 4).all()
    assert np.abs((W * ck ** 2 * ak).sum(0) - c ** 2 * a).max() > 1e-3


def test_bivariate_apply_equals_direct_sum_of_interpolated_symbol():
    """Linearity: sum_k w_k IDFT(q_k DFT v) equals the direct O(n^2) Op(q_M)
    with q_M(x, xi) = sum_k w_k(x) q_k(xi), here with an absorbing layer, a
    damping field independent of c, and both bases."""
    shape = (8, 6)
    c = np.ones(shape)
    c[2:6, 2:5] = 1.4
    c[3:5, 2:4] = 1.8
    zeta = np.zeros(shape)
    zeta[0, :] = 0.3
    zeta[:, 0] = 0.2
    zeta[0, 0] = 0.3
    a = 3.0 + rng(4).uniform(0, 6, shape)
    v = S.random_field(rng(5), shape)
    for basis, M in ((0, 3), (1, 5)):
        med = O.make_medium(c, zeta, a, 12.0, M=M, Mt=2, c_o=1.0, alpha=0.1, Ma=3, basis=basis)
        x = O.apply_preconditioner(med, v, exact=True)
        y = O.apply_pdo_direct(O.interpolated_symbol_at_point(med), v)
        np.testing.assert_allclose(x, y, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("basis", [0, 1])
def test_bivariate_exact_where_c_and_a_are_nodes(basis):
    """Where c(x) and a(x) take node values only, q_M(x, .) = q(x, .) and
    Q_M v equals the un-interpolated Op(q) with the point's own damping."""
    shape = (6, 8)
    r = rng(6)
    c = r.choice([1.0, 1.5, 2.0], size=shape)
    a = r.choice([2.0, 5.0, 8.0], size=shape)
    c[0, 0], c[0, 1], a[0, 0], a[0, 1] = 1.0, 2.0, 2.0, 8.0
    med = O.make_medium(c, None, a, 15.0, M=3, c_o=1.0, alpha=0.2, Ma=3, basis=basis)
    np.testing.assert_allclose(med.nodes.a_nodes, [2.0, 5.0, 8.0])
    v = S.random_field(r, shape)
    x = O.apply_preconditioner(med, v, exact=True)
    y = O.apply_pdo_direct(O.exact_symbol_at_point(med), v)
    np.testing.assert_allclose(x, y, atol=1e-12 * np.abs(x).max())


def test_bivariate_interpolation_converges_second_order_in_a():
    """Hats in a: ||(Q - Q_{Ma}) v|| falls like h_a^2 at fixed c (one speed
    node), the damping analogue of Thm. Acc."""
    shape = (12, 12)
    a = _independent_damping(shape)
    v = S.random_field(rng(8), shape)
    ref = None
    errs, hs = [], []
    for Ma in (3, 5, 9, 17):
        med = O.make_medium(np.ones(shape), None, a, 20.0, M=1, c_o=1.0, alpha=0.0, Ma=Ma)
        if ref is None:
            ref = O.apply_pdo_direct(O.exact_symbol_at_point(med), v)
        errs.append(np.linalg.norm(O.apply_preconditioner(med, v) - ref))
        hs.append((a.max() - a.min()) / (Ma - 1))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 1.8 < slope < 2.6, (errs, slope)


def test_bivariate_with_constant_damping_is_the_univariate_preconditioner():
    """A constant a collapses the damping nodes to one; the result is the
    univariate Q_M with a_node = that constant."""
    shape = (8, 8)
    c = _smooth_speed(shape)
    v = S.random_field(rng(9), shape)
    a = np.full(shape, 4.0)
    biv = O.make_medium(c, None, a, 20.0, M=5, c_o=1.0, alpha=0.1, Ma=4)
    uni = O.make_medium(c, None, a, 20.0, M=5, c_o=1.0, alpha=0.1, a_node=4.0)
    assert biv.nodes.K == uni.nodes.K == 5
    np.testing.assert_array_equal(O.apply_preconditioner(biv, v), O.apply_preconditioner(uni, v))
