"""Plain, slow, FP64 CPU oracle for the interpolated pseudodifferential
Helmholtz preconditioner of Acosta, Khajah & Palacios (arXiv 2409.16172).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
the tests, the smoke check and the CPU-baseline leg of the benchmark call it.
It shares no code with the CUDA path: the two meet only through the seeded
input arrays (wave speed, absorbing-layer profile, damping, right-hand side).

Everything here is complex128 / float64 and follows the paper's formulas in
the order the paper states them, with no blocking or fusion:

  * Helmholtz operator  c^2 Lap u + w^2 u + i w a u = f            (Eqn. 001)
  * operator symbol     p = w^2 + i w a - c^2 |xi|^2               (Eqn. 005)
  * principal symbol    q_{-2} = 1/p                               (Eqn. 021)
  * interpolated symbol q_M(c, xi) = sum_m phi_m(c) q(c_m, xi)     (Eqn. 105)
  * operator            Q_M v = sum_m phi_m(c(x)) IFT(q(c_m,.) FT v) (Eqn. 103)
  * complex wave speed  gamma = c (1 - i zeta)                     (Eqn. Complex_wave_speed)
  * layer interpolation real hats x zeta hats                      (Eqn. 405 / 403)
  * extensions the paper names as future work (Section 6): piecewise
    quadratic Lagrange bases in c, and bivariate interpolation in (c, a)
    with a independent of c (tensor products with hats in a)
  * discretisation      periodic 2nd-order central differences and
                        the FFT on the same grid                   (Section 5, Eqn. MainDiscrete)
  * solver              restarted GMRES, matrix-free               (Section 5, "GMRES implementation")

Readings of places where the paper is silent:
  * a = 0 in the operator is allowed; every node symbol carries the damping
    a_k = a_node + alpha * omega (alpha is a plan parameter).
  * |xi|^2 is the continuous (2 pi k / L)^2 by default (Eqn. 021); the
    finite-difference-consistent (4/h^2) sin^2(pi k / N) is an option.
  * Real nodes are equispaced on [c_min, c_max] (Lemma 3).  When an
    absorbing layer is present c_o must be a node (Section 4.4): if c_o lies
    strictly inside the range the M nodes are split into two equispaced
    segments in proportion to their lengths (at least one interval each).
  * Layer nodes are c_o (1 - i zeta_m), zeta_m = m zeta_max / Mt, m = 1..Mt;
    zeta_0 = 0 is the real node c_o.  Im(gamma) <= 0 (the '1 + i zeta_max'
    printed in Section 4.4 is read as a typo for 1 - i zeta_max).
  * Quadratic Lagrange basis (basis = 1): M odd, elements of two consecutive
    intervals [c_2e, c_2e+2], each segment of the two-segment split holding
    an even number of intervals; layer points keep the hats in zeta.
  * Cubic Hermite basis (basis = 2): on each interval the value planes take
    h00, h01 and extra planes with the symbol's derivative dq/dc at the two
    real nodes take h h10, h h11 (K = M + Mt + M planes); layer points keep
    the hats in zeta.
  * Bivariate interpolation (Ma >= 2): Ma damping nodes equispaced on
    [min a, max a]; node (s, j) carries gamma_s and damping a_j + alpha w;
    weights are products of the speed weights and hats in a.
  * DFT: unnormalised forward with e^{-2 pi i jk/N}, 1/n on the inverse;
    this is the discrete form of the symmetric pair in Eqn. FT.

What pins each function (tests/test_oracle_pins.py, tests/test_oracle_extensions.py; no
function here is "parity unpinned"):
  dft                     numpy.fft on 1D/2D/3D shapes; delta <-> constant, plane wave -> one
                          bin (fixes the sign), Parseval
  xi2_axis / xi2_grid     fftfreq order; the discrete table is minus the eigenvalue of the
                          periodic second difference
  apply_operator          plane-wave eigenfunction with gamma = c (1 - i zeta) and a > 0
                          (fixes the signs of zeta and of i w a); O(h^2) consistency
  real_nodes, build_nodes equispaced nodes, c_o a node, the two-segment split (and its
                          even-interval form for the quadratic basis)
  hat_weights             partition of unity, <= 2 non-zeros, reproduction of gamma (hats);
                          reproduction of 1, c, c^2 and <= 3 non-zeros (quadratic basis);
                          reproduction of cubics from values and derivatives, not of c^4,
                          <= 4 non-zeros (cubic Hermite)
  node_symbol_dc          central difference of node_symbol in c
  damping_nodes, damping_weights, interp_weights
                          reproduction of every bilinear f(c, a), <= 4 non-zeros, collapse to
                          the univariate form for constant a
  node_symbol             constant medium: Q_M is the Fourier multiplier of Eqn. 021; the
                          Lemma 3 bound with the printed second derivative
  apply_preconditioner    plane-wave closed form; equals the direct O(n^2) Op(q_M); equals the
                          un-interpolated Op(q) where the medium takes node values;
                          Q_{N,M} P_N = I (discrete symbol, constant c, a > 0, alpha = 0);
                          convergence orders 2 (hats, in c and in a), 3 (quadratic) and 4
                          (cubic Hermite)
  apply_pdo_direct, exact_symbol_at_point, interpolated_symbol_at_point
                          the constant-medium closed form and the pins above
  assemble_dense          column by column from apply_operator, then checked through the LU
                          solves below; the dense Q_M P_N spectrum gathers near 1 as M grows
                          and matches the un-interpolated Q P_N (Thms. 1-2, soft)
  gmres, givens           right and left forms equal dense LU; unpreconditioned GMRES too;
                          monotone Givens estimate within a cycle; preconditioning reduces the
                          step count; the paper's Example 1 residual gap
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

try:  # scipy.fft lets the CPU baseline use several host threads
    import scipy.fft as _sfft
except Exception:  # pragma: no cover
    _sfft = None


# ----------------------------------------------------------------------------
# Discrete Fourier transform (Section 2, Eqn. FT; Section 5: "FFT on the same
# grid").  Arrays are indexed [z][y][x] (x fastest); every axis is periodic.
# ----------------------------------------------------------------------------

def dft_matrix(N: int, sign: int) -> np.ndarray:
    """Dense N x N DFT matrix F[k, j] = exp(sign * 2 pi i (j k mod N) / N).

    The exponent is reduced modulo N in integers before the exp so that the
    matrix is accurate for any N.  Pinned by tests against numpy.fft and the
    delta / constant / plane-wave closed forms.
    """
    j = np.arange(N, dtype=np.int64)
    e = np.outer(j, j) % N
    return np.exp(sign * 2j * np.pi * e.astype(np.float64) / N)


def dft(v: np.ndarray, inverse: bool = False, exact: bool = False,
        workers: int = 1) -> np.ndarray:
    """d-dimensional DFT over every axis of v (the grid shape).

    forward: vhat[k] = sum_j v[j] exp(-2 pi i j.k / N)            (no scaling)
    inverse: v[j]    = (1/n) sum_k vhat[k] exp(+2 pi i j.k / N)

    exact=True uses the dense per-axis matrices ("oracle-exact");
    exact=False uses a library FFT ("oracle-fast").
    """
    v = np.asarray(v, dtype=np.complex128)
    if not exact:
        if _sfft is not None:
            return _sfft.ifftn(v, workers=workers) if inverse else _sfft.fftn(v, workers=workers)
        return np.fft.ifftn(v) if inverse else np.fft.fftn(v)
    out = v
    for ax in range(v.ndim):
        N = v.shape[ax]
        F = dft_matrix(N, +1 if inverse else -1)
        out = np.moveaxis(np.tensordot(F, out, axes=([1], [ax])), 0, ax)
        if inverse:
            out = out / N
    return out


def signed_index(N: int) -> np.ndarray:
    """Frequency index k' of each DFT bin k, in [-N/2, N/2) (numpy fftfreq order)."""
    k = np.arange(N)
    return np.where(k <= (N - 1) // 2, k, k - N)


def xi2_axis(N: int, L: float, symbol_kind: int = 0) -> np.ndarray:
    """Per-axis squared wavenumber table.

    symbol_kind 0: (2 pi k'/L)^2, the continuous |xi|^2 of Eqn. 005 / 021.
    symbol_kind 1: (4/h^2) sin^2(pi k/N), h = L/N, the symbol of the
                   second-order central difference of Section 5.
    """
    if symbol_kind == 0:
        kk = signed_index(N).astype(np.float64)
        return (2.0 * np.pi * kk / L) ** 2
    if symbol_kind == 1:
        h = L / N
        k = np.arange(N, dtype=np.float64)
        return (4.0 / h ** 2) * np.sin(np.pi * k / N) ** 2
    raise ValueError("symbol_kind must be 0 or 1")


def xi2_grid(shape, L: float, symbol_kind: int = 0) -> np.ndarray:
    """|xi|^2 on the whole frequency grid: the sum of the per-axis tables."""
    out = np.zeros(shape, dtype=np.float64)
    d = len(shape)
    for ax in range(d):
        t = xi2_axis(shape[ax], L, symbol_kind)
        bshape = [1] * d
        bshape[ax] = shape[ax]
        out = out + t.reshape(bshape)
    return out


# ----------------------------------------------------------------------------
# Medium (Section 3 assumptions; Section 4.4 absorbing layer)
# ----------------------------------------------------------------------------

def complex_speed(c: np.ndarray, zeta: np.ndarray) -> np.ndarray:
    """gamma = c (1 - i zeta)   (Eqn. Complex_wave_speed)."""
    return np.asarray(c, np.float64) * (1.0 - 1j * np.asarray(zeta, np.float64))


def validate_medium(c, zeta, c_o: float, rtol: float = 1e-12) -> None:
    """Section 3 needs 0 < c; Section 4.4 needs zeta >= 0 and c = c_o
    wherever zeta > 0 (so that the layer values lie on one vertical segment)."""
    c = np.asarray(c)
    zeta = np.asarray(zeta)
    if not np.all(np.isfinite(c)) or np.any(c <= 0):
        raise ValueError("wave speed must be finite and positive")
    if not np.all(np.isfinite(zeta)) or np.any(zeta < 0):
        raise ValueError("zeta must be finite and non-negative")
    lay = zeta > 0
    if np.any(np.abs(c[lay] - c_o) > rtol * c_o):
        raise ValueError("c must equal c_o inside the absorbing layer")


@dataclass
class Nodes:
    """Interpolation node table (Section 4.1 and 4.4).

    gamma[k]  complex node speed (real nodes first, then layer nodes)
    a[k]      damping used in node k's symbol
    c_real    the M_eff real nodes, increasing
    zeta_nodes zeta_0 = 0 < zeta_1 < ... < zeta_Mt
    m_o       index of c_o among the real nodes (-1 when there is no layer)
    a_nodes   damping nodes of the bivariate form (one entry otherwise);
              node k = s * Ma + j has speed node s and damping node j
    basis     0: piecewise-linear hats in c; 1: piecewise quadratic Lagrange;
              2: piecewise cubic Hermite (value and c-derivative planes)
    deriv     per node: 0 for the symbol q(gamma_k, xi), 1 for its derivative
              in the wave speed dq/dc at the real node c_k (basis 2)
    """
    gamma: np.ndarray
    a: np.ndarray
    c_real: np.ndarray
    zeta_nodes: np.ndarray
    m_o: int
    omega: float
    a_nodes: np.ndarray = field(default_factory=lambda: np.zeros(1))
    basis: int = 0
    alpha: float = 0.05
    deriv: np.ndarray = field(default=None)

    @property
    def K(self) -> int:
        return len(self.gamma)

    @property
    def Ma(self) -> int:
        return len(self.a_nodes)

    @property
    def Ks(self) -> int:
        """Number of speed nodes (real and layer)."""
        return self.K // self.Ma

    @property
    def M(self) -> int:
        return len(self.c_real)

    @property
    def Mt(self) -> int:
        return len(self.zeta_nodes) - 1


def real_nodes(c_lo: float, c_hi: float, M: int, c_o: float | None,
               basis: int = 0) -> np.ndarray:
    """Equispaced real nodes with c_1 = c_lo and c_M = c_hi (Lemma 3).

    If c_o is given it must be a node (Section 4.4): when it lies strictly
    inside (c_lo, c_hi) the range is split at c_o into two equispaced
    segments; segment 1 gets s1 = clamp(round((M-1)(c_o-c_lo)/(c_hi-c_lo)),
    1, M-2) intervals.  M = 1 gives the single node c_o (or c_lo), i.e. the
    Q_1 preconditioner of Eqn. OneInterpPoint.  A range narrower than
    1e-12 c_hi also collapses to one node.

    basis = 1 (quadratic elements of two intervals) needs M odd, and the
    split gives each segment an even number of intervals:
    s1 = clamp(2 round((M-1)(c_o-c_lo)/(2(c_hi-c_lo))), 2, M-3).
    """
    if M < 1:
        raise ValueError("M must be >= 1")
    if M == 1:
        return np.array([c_o if c_o is not None else c_lo], dtype=np.float64)
    if c_hi - c_lo <= 1e-12 * c_hi:
        return np.array([c_lo], dtype=np.float64)
    if basis == 1 and M % 2 == 0:
        raise ValueError("the quadratic basis needs an odd number of real nodes")
    if c_o is not None and c_lo < c_o < c_hi:
        if M < (5 if basis == 1 else 3):
            raise ValueError("c_o strictly inside the speed range needs more nodes")
        if basis == 1:
            s1 = 2 * int(math.floor((M - 1) * (c_o - c_lo) / (2.0 * (c_hi - c_lo)) + 0.5))
            s1 = min(max(s1, 2), M - 3)
        else:
            s1 = int(math.floor((M - 1) * (c_o - c_lo) / (c_hi - c_lo) + 0.5))
            s1 = min(max(s1, 1), M - 2)
        s2 = (M - 1) - s1
        left = [c_lo + (c_o - c_lo) * i / s1 for i in range(s1)]
        right = [c_o + (c_hi - c_o) * i / s2 for i in range(s2)]
        return np.array(left + right + [c_hi], dtype=np.float64)
    return np.array([c_lo + (c_hi - c_lo) * i / (M - 1) for i in range(M - 1)] + [c_hi],
                    dtype=np.float64)


def damping_nodes(a_lo: float, a_hi: float, Ma: int) -> np.ndarray:
    """Ma equispaced damping nodes on [a_lo, a_hi] (the second variable of
    the bivariate form); a range narrower than 1e-12 max(|a_hi|, 1)
    collapses to one node."""
    if Ma < 1:
        raise ValueError("Ma must be >= 1")
    if Ma == 1 or a_hi - a_lo <= 1e-12 * max(abs(a_hi), 1.0):
        return np.array([a_lo], dtype=np.float64)
    return np.array([a_lo + (a_hi - a_lo) * j / (Ma - 1) for j in range(Ma - 1)] + [a_hi],
                    dtype=np.float64)


def build_nodes(c, zeta, omega: float, M: int, Mt: int, c_o: float,
                zeta_max: float | None = None, alpha: float = 0.05,
                a_node: float = 0.0, a=None, Ma: int = 1, basis: int = 0) -> Nodes:
    """Node table of Section 4.1 / 4.4 for a given medium.

    Real nodes span [min c, max c] (c_o included when there is a layer);
    layer nodes are c_o (1 - i zeta_m), zeta_m = m zeta_max / Mt.
    zeta_max defaults to max(zeta).  With Ma <= 1 every node symbol uses the
    damping a_k = a_node + alpha * omega.  With Ma >= 2 the damping a(x) is
    a second interpolation variable: node (s, j) (k = s Ma + j) uses speed
    node s and the damping a_j + alpha * omega, a_j equispaced on
    [min a, max a].
    """
    c = np.asarray(c, np.float64)
    zeta = np.asarray(zeta, np.float64)
    has_layer = bool(np.any(zeta > 0)) and Mt > 0
    c_lo, c_hi = float(c.min()), float(c.max())
    if has_layer:
        c_lo, c_hi = min(c_lo, c_o), max(c_hi, c_o)
    if basis == 2 and Ma >= 2:
        raise ValueError("the cubic Hermite basis is univariate (Ma <= 1)")
    cr = real_nodes(c_lo, c_hi, M, c_o if (has_layer or M == 1) else None,
                    1 if basis == 1 else 0)
    m_o = -1
    if has_layer:
        hit = np.nonzero(cr == c_o)[0]
        if len(hit) != 1:
            raise ValueError("c_o is not a node")
        m_o = int(hit[0])
        zmax = float(zeta.max()) if (zeta_max is None or zeta_max <= 0) else float(zeta_max)
        if zmax < float(zeta.max()):
            raise ValueError("zeta_max below the largest zeta of the medium")
        zn = np.array([0.0] + [m * zmax / Mt for m in range(1, Mt)] + [zmax])
    else:
        zn = np.array([0.0])
    gam_s = [complex(x) for x in cr] + [c_o * (1.0 - 1j * z) for z in zn[1:]]
    if Ma >= 2:
        av = np.zeros_like(c) if a is None else np.asarray(a, np.float64)
        an = damping_nodes(float(av.min()), float(av.max()), Ma)
    else:
        an = np.array([a_node], dtype=np.float64)
    gam = np.array([g for g in gam_s for _ in an], np.complex128)
    ak = np.array([aj + alpha * omega for _ in gam_s for aj in an], np.float64)
    deriv = np.zeros(len(gam), dtype=np.int64)
    if basis == 2 and len(cr) >= 2:
        # cubic Hermite: one derivative plane dq/dc per real node, after the
        # value planes
        gam = np.concatenate([gam, cr.astype(np.complex128)])
        ak = np.concatenate([ak, np.full(len(cr), an[0] + alpha * omega)])
        deriv = np.concatenate([deriv, np.ones(len(cr), dtype=np.int64)])
    return Nodes(gam, ak, cr, zn, m_o, float(omega), an, int(basis), float(alpha), deriv)


def hat_weights(c, zeta, nodes: Nodes) -> np.ndarray:
    """Dense speed weights W[s, x] of Eqn. 405 (s over the Ks speed nodes):
    piecewise-linear hats, or with nodes.basis == 1 quadratic Lagrange
    polynomials on the real elements (layer points keep hats in zeta).

    Points with zeta = 0 get the real hats phi_m(c(x)) on the real nodes.
    Points with zeta > 0 (where c = c_o) get phi_0(Im gamma) on node m_o and
    phi_m(Im gamma) on layer node m; the hats in Im gamma = -c_o zeta are the
    hats in zeta because the map is linear.  At most two weights per point
    are non-zero and they sum to one.
    """
    c = np.asarray(c, np.float64)
    zeta = np.asarray(zeta, np.float64)
    cf, zf = c.ravel(), zeta.ravel()
    W = np.zeros((nodes.Ks, cf.size), dtype=np.float64)
    real = np.nonzero(zf == 0)[0]
    cr = nodes.c_real
    M = len(cr)
    if M == 1:
        W[0, real] = 1.0
    elif len(real) and nodes.basis == 2:
        # cubic Hermite on [c_i, c_{i+1}], t = (c - c_i) / h: the values
        # take h00 = 2t^3 - 3t^2 + 1 and h01 = 3t^2 - 2t^3, the derivative
        # planes h h10 = h (t^3 - 2t^2 + t) and h h11 = h (t^3 - t^2)
        cv = cf[real]
        i = np.clip(np.searchsorted(cr, cv, side="right") - 1, 0, M - 2)
        h = cr[i + 1] - cr[i]
        t = (cv - cr[i]) / h
        if np.any(t < -1e-12) or np.any(t > 1 + 1e-12):
            raise ValueError("wave speed outside the node range")
        nv = len(nodes.gamma) - M  # value planes come first
        np.add.at(W, (i, real), 2 * t ** 3 - 3 * t ** 2 + 1)
        np.add.at(W, (i + 1, real), 3 * t ** 2 - 2 * t ** 3)
        np.add.at(W, (nv + i, real), h * (t ** 3 - 2 * t ** 2 + t))
        np.add.at(W, (nv + i + 1, real), h * (t ** 3 - t ** 2))
    elif len(real) and nodes.basis == 1:
        # element e spans the nodes 2e, 2e+1, 2e+2; Lagrange polynomials of
        # degree 2 through them
        cv = cf[real]
        i = np.clip(np.searchsorted(cr, cv, side="right") - 1, 0, M - 2)
        e = np.minimum(i // 2, (M - 1) // 2 - 1)
        if np.any(cv < cr[0] - 1e-12 * cr[-1]) or np.any(cv > cr[-1] * (1 + 1e-12)):
            raise ValueError("wave speed outside the node range")
        n0, n1, n2 = 2 * e, 2 * e + 1, 2 * e + 2
        c0, c1, c2 = cr[n0], cr[n1], cr[n2]
        np.add.at(W, (n0, real), (cv - c1) * (cv - c2) / ((c0 - c1) * (c0 - c2)))
        np.add.at(W, (n1, real), (cv - c0) * (cv - c2) / ((c1 - c0) * (c1 - c2)))
        np.add.at(W, (n2, real), (cv - c0) * (cv - c1) / ((c2 - c0) * (c2 - c1)))
    elif len(real):
        cv = cf[real]
        i = np.clip(np.searchsorted(cr, cv, side="right") - 1, 0, M - 2)
        t = (cv - cr[i]) / (cr[i + 1] - cr[i])
        if np.any(t < -1e-12) or np.any(t > 1 + 1e-12):
            raise ValueError("wave speed outside the node range")
        np.add.at(W, (i, real), 1.0 - t)
        np.add.at(W, (i + 1, real), t)
    lay = np.nonzero(zf > 0)[0]
    if len(lay):
        zn = nodes.zeta_nodes
        Mt = len(zn) - 1
        if Mt < 1:
            raise ValueError("layer present but no layer nodes")
        zv = zf[lay]
        i = np.clip(np.searchsorted(zn, zv, side="right") - 1, 0, Mt - 1)
        t = (zv - zn[i]) / (zn[i + 1] - zn[i])
        if np.any(t > 1 + 1e-12):
            raise ValueError("zeta above zeta_max")
        node_of = np.array([nodes.m_o] + [M + m - 1 for m in range(1, Mt + 1)])
        np.add.at(W, (node_of[i], lay), 1.0 - t)
        np.add.at(W, (node_of[i + 1], lay), t)
    return W.reshape((nodes.Ks,) + c.shape)


def damping_weights(a, nodes: Nodes) -> np.ndarray:
    """Dense hats Wa[j, x] of a(x) on the damping nodes (all ones for a
    single damping node)."""
    av = np.asarray(a, np.float64).ravel()
    an = nodes.a_nodes
    Wa = np.zeros((len(an), av.size), dtype=np.float64)
    if len(an) == 1:
        Wa[0] = 1.0
    else:
        j = np.clip(np.searchsorted(an, av, side="right") - 1, 0, len(an) - 2)
        t = (av - an[j]) / (an[j + 1] - an[j])
        if np.any(t < -1e-12) or np.any(t > 1 + 1e-12):
            raise ValueError("damping outside the node range")
        idx = np.arange(av.size)
        np.add.at(Wa, (j, idx), 1.0 - t)
        np.add.at(Wa, (j + 1, idx), t)
    return Wa.reshape((len(an),) + np.shape(a))


def interp_weights(c, zeta, a, nodes: Nodes) -> np.ndarray:
    """Weights W[k, x] of node k = s Ma + j: speed weight of node s times the
    damping hat of node j (the tensor-product form of Eqn. 405 in (c, a))."""
    Ws = hat_weights(c, zeta, nodes)
    Wa = damping_weights(a, nodes)
    W = np.zeros((nodes.K,) + np.shape(c), dtype=np.float64)
    for s_ in range(nodes.Ks):
        for j in range(nodes.Ma):
            W[s_ * nodes.Ma + j] = Ws[s_] * Wa[j]
    return W


def node_symbol(gamma_k: complex, a_k: float, omega: float, xi2: np.ndarray) -> np.ndarray:
    """q(gamma_k, xi) = 1 / (w^2 + i w a_k - gamma_k^2 |xi|^2)   (Eqn. 021 with c -> gamma)."""
    return 1.0 / (omega ** 2 + 1j * omega * a_k - gamma_k ** 2 * xi2)


def node_symbol_dc(c_k: float, a_k: float, omega: float, xi2: np.ndarray) -> np.ndarray:
    """dq/dc at the real node c_k: with q = 1/p, p = w^2 + i w a - c^2 |xi|^2
    (Eqn. 021), dq/dc = -p_c / p^2 = 2 c |xi|^2 / p^2 (the first derivative
    in c of the symbol whose second derivative Section 4.3 prints)."""
    p = omega ** 2 + 1j * omega * a_k - c_k ** 2 * xi2
    return 2.0 * c_k * xi2 / p ** 2


def symbol_of(nodes: Nodes, k: int, omega: float, xi2: np.ndarray) -> np.ndarray:
    """The symbol of plane k: q(gamma_k, xi), or dq/dc for a derivative plane."""
    if nodes.deriv is not None and nodes.deriv[k]:
        return node_symbol_dc(float(nodes.gamma[k].real), nodes.a[k], omega, xi2)
    return node_symbol(nodes.gamma[k], nodes.a[k], omega, xi2)


# ----------------------------------------------------------------------------
# Preconditioner apply (Eqn. 103 / 403): one forward DFT, K symbol multiplies
# each followed by an inverse DFT, then the pointwise weighted sum.
# ----------------------------------------------------------------------------

@dataclass
class Medium:
    """Everything the oracle needs about one problem instance."""
    c: np.ndarray
    zeta: np.ndarray
    a: np.ndarray            # damping in the operator (Eqn. 001)
    omega: float
    L: float
    nodes: Nodes
    W: np.ndarray            # dense hat weights, shape (K,) + grid
    symbol_kind: int = 0
    xi2: np.ndarray = field(default=None)

    @property
    def shape(self):
        return self.c.shape

    @property
    def gamma2(self) -> np.ndarray:
        return complex_speed(self.c, self.zeta) ** 2


def make_medium(c, zeta=None, a=None, omega: float = 1.0, M: int = 8, Mt: int = 0,
                c_o: float = 1.0, zeta_max: float | None = None, alpha: float = 0.05,
                a_node: float = 0.0, symbol_kind: int = 0, L: float = 1.0, Ma: int = 1,
                basis: int = 0) -> Medium:
    """Validate a medium and build its node table and weights."""
    c = np.asarray(c, np.float64)
    zeta = np.zeros_like(c) if zeta is None else np.asarray(zeta, np.float64)
    a = np.zeros_like(c) if a is None else np.asarray(a, np.float64)
    validate_medium(c, zeta, c_o)
    nodes = build_nodes(c, zeta, omega, M, Mt, c_o, zeta_max, alpha, a_node, a, Ma, basis)
    W = interp_weights(c, zeta, a, nodes)
    return Medium(c, zeta, a, float(omega), float(L), nodes, W, symbol_kind,
                  xi2_grid(c.shape, L, symbol_kind))


def apply_preconditioner(med: Medium, v: np.ndarray, exact: bool = False,
                         workers: int = 1) -> np.ndarray:
    """Q_M v = sum_k w_k(x) * IDFT( q_k(xi) * DFT(v) )   (Eqn. 103 / 403)."""
    vhat = dft(v, inverse=False, exact=exact, workers=workers)
    out = np.zeros(med.shape, dtype=np.complex128)
    for k in range(med.nodes.K):
        qk = symbol_of(med.nodes, k, med.omega, med.xi2)
        uk = dft(qk * vhat, inverse=True, exact=exact, workers=workers)
        out += med.W[k] * uk
    return out


def apply_pdo_direct(symbol_at_point, v: np.ndarray, L: float = 1.0,
                     symbol_kind: int = 0) -> np.ndarray:
    """Direct O(n^2) evaluation of Op(q) v on the grid (Eqn. GeneralPSDO,
    Eqn. Precond):  (Op(q) v)(x_j) = (1/n) sum_k q(x_j, xi_k) vhat_k e^{2 pi i j.k/N}.

    symbol_at_point(flat_index, xi2_flat) -> q over all frequencies for that
    point.  Only for tiny grids (n <= ~1024).
    """
    shape = v.shape
    n = v.size
    vhat = dft(v, exact=True).ravel()
    xi2 = xi2_grid(shape, L, symbol_kind).ravel()
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    jidx = [g.ravel() for g in grids]
    out = np.zeros(n, dtype=np.complex128)
    for p in range(n):
        ph = np.zeros(n, dtype=np.float64)
        for ax, N in enumerate(shape):
            ph = ph + ((jidx[ax][p] * jidx[ax]) % N) / N
        e = np.exp(2j * np.pi * ph)
        q = symbol_at_point(p, xi2)
        out[p] = np.sum(q * vhat * e) / n
    return out.reshape(shape)


def exact_symbol_at_point(med: Medium):
    """q_{-2}(gamma(x), xi) with the point's own complex speed (Eqn. Precond,
    the un-interpolated preconditioner Q); in the bivariate form also with
    the point's own damping a(x) + alpha * omega."""
    g = complex_speed(med.c, med.zeta).ravel()
    if med.nodes.Ma >= 2:
        damp = med.a.ravel() + med.nodes.alpha * med.omega
    else:
        damp = np.full(g.size, med.nodes.a[0])

    def f(p, xi2):
        return 1.0 / (med.omega ** 2 + 1j * med.omega * damp[p] - g[p] ** 2 * xi2)
    return f


def interpolated_symbol_at_point(med: Medium):
    """q_M(gamma(x), xi) = sum_k w_k(x) q(gamma_k, xi)   (Eqn. 105 / 405)."""
    Wf = med.W.reshape(med.nodes.K, -1)

    def f(p, xi2):
        s = np.zeros_like(xi2, dtype=np.complex128)
        for k in range(med.nodes.K):
            if Wf[k, p] != 0.0:
                s = s + Wf[k, p] * symbol_of(med.nodes, k, med.omega, xi2)
        return s
    return f


# ----------------------------------------------------------------------------
# Finite-difference Helmholtz operator P_N (Eqn. 001 discretised as in
# Section 5: second-order centred differences, periodic boundaries).
# ----------------------------------------------------------------------------

def apply_operator(med: Medium, u: np.ndarray) -> np.ndarray:
    """(P_N u)_j = gamma_j^2 sum_axes (u_{j+e} - 2 u_j + u_{j-e}) / h_axis^2
                   + (w^2 + i w a_j) u_j,  h_axis = L / N_axis, periodic."""
    u = np.asarray(u, np.complex128)
    lap = np.zeros_like(u)
    for ax in range(u.ndim):
        h = med.L / u.shape[ax]
        lap += (np.roll(u, -1, axis=ax) - 2.0 * u + np.roll(u, 1, axis=ax)) / h ** 2
    return med.gamma2 * lap + (med.omega ** 2 + 1j * med.omega * med.a) * u


def assemble_dense(apply_fn, shape) -> np.ndarray:
    """Dense n x n matrix of a linear grid operator, column by column."""
    n = int(np.prod(shape))
    A = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1.0
        A[:, j] = apply_fn(e.reshape(shape)).ravel()
    return A


# ----------------------------------------------------------------------------
# Restarted GMRES with CGS2 Arnoldi and complex Givens rotations
# (Section 5 "GMRES implementation"; right / flexible preconditioning).
# ----------------------------------------------------------------------------

def givens(a: complex, b: complex):
    """Rotation G = [[c, s], [-conj(s), c]] with c real and G [a, b]^T = [r, 0]^T."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, np.conj(b) / abs(b), abs(b) + 0j
    rho = math.hypot(abs(a), abs(b))
    c = abs(a) / rho
    s = (a / abs(a)) * np.conj(b) / rho
    r = (a / abs(a)) * rho
    return c, s, r


def gmres(apply_A, f: np.ndarray, apply_M=None, restart: int = 30, tol: float = 1e-6,
          maxit: int = 4000, x0: np.ndarray | None = None, side: str = "right",
          record_history: bool = False):
    """Restarted GMRES(m).

    side='right': flexible right preconditioning (FGMRES): z_j = M v_j is
      stored and x += Z y at the end of a cycle.  The stopping test is on the
      true relative residual ||f - A x|| / ||f|| <= tol, checked with the
      operator after every cycle whose Givens estimate reached tol.
    side='left': the paper's (Q P) u = Q f form (Eqn. MainDiscretePrecond),
      stopping on the preconditioned residual; kept for comparison.

    Arnoldi uses classical Gram-Schmidt applied twice (CGS2).
    Returns (x, stats) with stats = dict(iters, restarts, rel_true_resid,
    converged, history).
    """
    f = np.asarray(f, np.complex128)
    shape = f.shape
    n = f.size
    M_ = apply_M if apply_M is not None else (lambda v: v)
    x = np.zeros(n, np.complex128) if x0 is None else np.asarray(x0, np.complex128).ravel().copy()

    def A(v):
        return apply_A(v.reshape(shape)).ravel()

    def Mv(v):
        return M_(v.reshape(shape)).ravel()

    if side == "left":
        b = Mv(f.ravel())

        def op(v):
            return Mv(A(v))
    else:
        b = f.ravel()
        op = None
    bnorm = np.linalg.norm(b)
    fnorm = np.linalg.norm(f)
    history = []
    iters = 0
    restarts = 0
    if bnorm == 0:
        return x.reshape(shape), dict(iters=0, restarts=0, rel_true_resid=0.0,
                                      converged=True, history=history)
    converged = False
    while iters < maxit:
        r = b - (op(x) if side == "left" else A(x))
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            converged = True
            break
        m = restart
        V = np.zeros((m + 1, n), np.complex128)
        Z = np.zeros((m, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            if side == "left":
                w = op(V[j])
            else:
                Z[j] = Mv(V[j])
                w = A(Z[j])
            # CGS2: two passes of classical Gram-Schmidt
            h1 = V[:j + 1].conj() @ w
            w = w - V[:j + 1].T @ h1
            h2 = V[:j + 1].conj() @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h1 + h2
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            iters += 1
            breakdown = hn <= 1e-14 * max(abs(H[:j + 1, j]).max(), 1e-300)
            if not breakdown:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c_, s_, r_ = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c_, s_
            H[j, j] = r_
            H[j + 1, j] = 0
            g[j + 1] = -np.conj(s_) * g[j]
            g[j] = c_ * g[j]
            est = abs(g[j + 1]) / bnorm
            if record_history:
                history.append(est)
            j_end = j + 1
            if est <= tol or breakdown or iters >= maxit:
                break
        y = np.zeros(j_end, np.complex128)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_end] @ y[i + 1:j_end]) / H[i, i]
        if side == "left":
            x = x + V[:j_end].T @ y
        else:
            x = x + Z[:j_end].T @ y
        restarts += 1
    rt = np.linalg.norm(f.ravel() - A(x)) / fnorm
    if side == "right":
        converged = rt <= tol
    return x.reshape(shape), dict(iters=iters, restarts=restarts, rel_true_resid=float(rt),
                                  converged=bool(converged), history=history)
