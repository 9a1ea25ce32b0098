"""Seeded synthetic inputs: wave-speed media, absorbing-layer profiles and
right-hand sides.

This module is the only piece the CUDA path and the CPU oracle share.  It
draws and shapes input arrays only; it holds none of the method's arithmetic
(no symbols, nodes, weights, transforms, stencils or solvers).

Grid convention: the unit box [-L/2, L/2)^d with N points per axis,
x_j = -L/2 + j h, h = L / N, arrays indexed [z][y][x] (x fastest), periodic.

Media follow the workload recipes below; every random draw comes from
numpy's PCG64 seeded per workload.
  * Gaussian bumps c = 1 + A * sum exp(-|x - x_i|^2 / (2 sigma^2)) (2D/3D).
  * Horizontal layers smoothed with the paper's smooth Heaviside
    H_eta(s) = 1/(1 + exp(-s/eta)) (Section 5.1, Eqn. WS) plus spherical
    inclusions.
  * Absorbing layer of W cells on every face: zeta = zeta_max (W - d)/W at
    cell distance d < W from the nearest face (a linear ramp like Eqn. Zeta).
  * Because the interpolation needs c = c_o inside the layer (Section 4.4),
    every medium is blended to c_o by a raised-cosine taper over the 8 cells
    just inside the layer: c = c_o + tau (c_raw - c_o).
  * omega is set from points per wavelength at the slowest speed:
    PPW = 2 pi c_min N / (L omega) (Section 5.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TAPER_CELLS = 8


def coords(shape, L: float = 1.0):
    """Cell coordinates x_j = -L/2 + j L/N per axis, broadcastable to shape."""
    d = len(shape)
    out = []
    for ax, N in enumerate(shape):
        x = -L / 2 + np.arange(N) * (L / N)
        b = [1] * d
        b[ax] = N
        out.append(x.reshape(b))
    return out  # [z?, y, x] order follows the array axes


def face_distance(shape) -> np.ndarray:
    """Distance in cells from each cell to the nearest face of the box."""
    d = None
    for ax, N in enumerate(shape):
        i = np.arange(N)
        di = np.minimum(i, N - 1 - i)
        b = [1] * len(shape)
        b[ax] = N
        di = di.reshape(b)
        d = di if d is None else np.minimum(d, di)
    return np.broadcast_to(d, shape).astype(np.int64)


def layer_profile(shape, width: int, zeta_max: float) -> np.ndarray:
    """zeta = zeta_max (W - d) / W for d < W cells from the nearest face, else 0."""
    d = face_distance(shape)
    z = np.where(d < width, zeta_max * (width - d) / max(width, 1), 0.0)
    return z.astype(np.float64)


def taper(shape, width: int, cells: int = TAPER_CELLS) -> np.ndarray:
    """Raised-cosine blend factor: 0 in the layer, rising to 1 over the
    `cells` cells just inside it, 1 in the interior."""
    d = face_distance(shape)
    s = (d - width + 1) / (cells + 1)
    tau = np.where(d < width, 0.0,
                   np.where(d >= width + cells, 1.0, 0.5 * (1.0 - np.cos(np.pi * s))))
    return tau.astype(np.float64)


def omega_for_ppw(c_min: float, N: int, ppw: float, L: float = 1.0) -> float:
    """omega with PPW = 2 pi c_min N / (L omega) points per wavelength."""
    return 2.0 * math.pi * c_min * N / (ppw * L)


def smooth_heaviside(s, eta: float):
    """H_eta(s) = 1 / (1 + exp(-s / eta))  (Section 5.1, Eqn. WS)."""
    return 0.5 * (1.0 + np.tanh(np.asarray(s) / (2.0 * eta)))


@dataclass
class Problem:
    """One synthetic Helmholtz problem (inputs only)."""
    name: str
    shape: tuple
    c: np.ndarray
    zeta: np.ndarray
    a: np.ndarray | None
    omega: float
    c_o: float
    M: int
    Mt: int
    f: np.ndarray                 # (nrhs,) + shape, complex128
    restart: int = 40
    tol: float = 1e-6
    precision: int = 1            # 0 = FP64 plain path, 1 = c64 preconditioner
    layer_width: int = 0
    L: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    @property
    def K(self) -> int:
        return (self.M + self.Mt) * max(int(self.meta.get("Ma", 1)), 1)


def point_sources(rng, shape, width: int, nrhs: int) -> np.ndarray:
    """nrhs unit point sources f = e_j, j uniform among cells at least
    width + TAPER_CELLS cells from every face."""
    d = face_distance(shape).ravel()
    ok = np.nonzero(d >= width + TAPER_CELLS)[0]
    if len(ok) == 0:
        ok = np.arange(d.size)
    js = rng.choice(ok, size=nrhs, replace=nrhs > len(ok))
    f = np.zeros((nrhs, int(np.prod(shape))), np.complex128)
    f[np.arange(nrhs), js] = 1.0
    return f.reshape((nrhs,) + tuple(shape))


def bumps(rng, shape, n_bumps: int, amp, sigma, width: int, L: float = 1.0,
          margin_sigmas: float = 2.0):
    """Sum of Gaussian bumps; centres uniform in the interior box that keeps
    them margin_sigmas * sigma away from the taper zone (the whole interior
    when that box is empty)."""
    X = coords(shape, L)
    h = L / shape[-1]
    half_in = L / 2 - (width + TAPER_CELLS) * h
    out = np.zeros(shape, np.float64)
    for _ in range(n_bumps):
        a = amp(rng) if callable(amp) else amp
        s = sigma(rng) if callable(sigma) else sigma
        r = max(half_in - margin_sigmas * s, 0.0)
        ctr = rng.uniform(-r, r, size=len(shape)) if r > 0 else np.zeros(len(shape))
        d2 = sum((X[ax] - ctr[ax]) ** 2 for ax in range(len(shape)))
        out = out + a * np.exp(-d2 / (2 * s * s))
    return out


def finish_medium(c_raw, width, zeta_max, c_o=1.0, taper_cells: int = TAPER_CELLS):
    """Blend c_raw to c_o towards the layer and build the layer profile."""
    tau = taper(c_raw.shape, width, taper_cells)
    c = c_o + tau * (c_raw - c_o)
    zeta = layer_profile(c_raw.shape, width, zeta_max)
    return c, zeta


# ---------------------------------------------------------------------------
# The workloads
# ---------------------------------------------------------------------------

DEFAULT_ZETA_MAX = 0.15


def bump_problem(N: int, seed: int, *, d: int = 2, n_bumps: int = 3, amp=0.3,
                 sigma=0.1, width: int = 16, ppw: float = 10.0, M: int = 6, Mt: int = 2,
                 nrhs: int = 1, restart: int = 30, precision: int = 0,
                 zeta_max: float = DEFAULT_ZETA_MAX, name: str = "bumps") -> Problem:
    """c = 1 + amp * sum of Gaussian bumps (width sigma), unit box, a = 0,
    W-cell absorbing layer, omega for PPW points per wavelength at c_min."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (N,) * d
    c_raw = 1.0 + bumps(rng, shape, n_bumps, amp, sigma, width)
    c, zeta = finish_medium(c_raw, width, zeta_max)
    omega = omega_for_ppw(float(c.min()), N, ppw)
    f = point_sources(rng, shape, width, nrhs)
    return Problem(name, shape, c, zeta, None, omega, 1.0, M, Mt, f, restart,
                   1e-6, precision, width)


def config1(seed: int = 16173) -> Problem:
    """2D 128^2, c = 1 + 0.3 * (3 Gaussian bumps, sigma 0.1), a = 0,
    16-cell layer, 10 PPW, K = 8 (6 + 2), GMRES(30), FP64 throughout."""
    return bump_problem(128, seed, n_bumps=3, amp=0.3, sigma=0.1, width=16, ppw=10.0,
                        M=6, Mt=2, restart=30, precision=0, name="2d-128-bumps3-K8")


def config2(seed: int = 16174) -> Problem:
    """2D 1024^2, c in [1, 2] from 20 Gaussian bumps (amplitude U[0,1], sigma
    U[0.02,0.1]) plus the linear gradient 0.5 (x_1 + 1/2), mapped affinely to
    [1, 2]; 32-cell layer, 8 PPW, K = 16 (12 + 4), FGMRES(40), c64 apply."""
    N, width = 1024, 32
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (N, N)
    raw = bumps(rng, shape, 20, lambda r: r.uniform(0, 1), lambda r: r.uniform(0.02, 0.1),
                width)
    X = coords(shape)
    raw = raw + 0.5 * (X[1] + 0.5)
    raw = 1.0 + (raw - raw.min()) / (raw.max() - raw.min())
    c, zeta = finish_medium(raw, width, DEFAULT_ZETA_MAX)
    omega = omega_for_ppw(float(c.min()), N, 8.0)
    f = point_sources(rng, shape, width, 1)
    return Problem("2d-1024-bumps20-grad-K16", shape, c, zeta, None, omega, 1.0, 12, 4, f,
                   40, 1e-6, 1, width)


def config3(seed: int = 16175, N: int = 256) -> Problem:
    """3D N^3 (256 by default), 6 horizontal layers with speeds U[1,3] and
    seeded interface depths smoothed by H_eta (eta = 2h), 10 spherical
    inclusions of radius 8-20 cells with contrast +-20%; 24-cell layer,
    8 PPW at c_min, K = 16 (12 + 4), FGMRES(40), c64 apply."""
    width = 24 if N >= 128 else max(4, N // 10)
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (N, N, N)
    Z, Y, X = coords(shape)
    h = 1.0 / N
    eta = 2 * h
    speeds = rng.uniform(1.0, 3.0, size=6)
    depths = np.sort(rng.uniform(-0.5 + (width + TAPER_CELLS) * h,
                                 0.5 - (width + TAPER_CELLS) * h, size=5))
    raw = np.full(shape, speeds[0])
    for i, zi in enumerate(depths):
        raw = raw + (speeds[i + 1] - speeds[i]) * smooth_heaviside(Z - zi, eta)
    half_in = 0.5 - (width + TAPER_CELLS) * h
    for _ in range(10):
        r = rng.uniform(8, 20) * (N / 256.0) * h
        sgn = 1.0 if rng.uniform() < 0.5 else -1.0
        ctr = rng.uniform(-max(half_in - r, 0), max(half_in - r, 0), size=3)
        dist = np.sqrt((Z - ctr[0]) ** 2 + (Y - ctr[1]) ** 2 + (X - ctr[2]) ** 2)
        raw = raw * (1.0 + 0.2 * sgn * smooth_heaviside(r - dist, eta))
    c, zeta = finish_medium(raw, width, DEFAULT_ZETA_MAX)
    omega = omega_for_ppw(float(c.min()), N, 8.0)
    f = point_sources(rng, shape, width, 1)
    return Problem(f"3d-{N}-layers6-incl10-K16", shape, c, zeta, None, omega, 1.0, 12, 4, f,
                   40, 1e-6, 1, width)


def config4(seed: int = 16176, nrhs: int = 64, N: int = 512) -> Problem:
    """2D 512^2 shared medium from the 128^2 recipe, 64 point sources,
    K = 12 (9 + 3), FGMRES(40) per right-hand side, c64 apply."""
    p = bump_problem(N, seed, n_bumps=3, amp=0.3, sigma=0.1, width=16, ppw=10.0, M=9, Mt=3,
                     nrhs=nrhs, restart=40, precision=1, name=f"2d-{N}-bumps3-K12-{nrhs}rhs")
    return p


SERVING_GRIDS = [(256, 256), (512, 512), (1024, 1024), (2048, 2048),
                 (64, 64, 64), (128, 128, 128), (192, 192, 192)]


def serving_request(rng, grids=SERVING_GRIDS, max_rhs: int = 8) -> Problem:
    """One request of the serving stream: a grid drawn uniformly from the
    list, 6-12 PPW, a Gaussian-bump medium mapped to c in [1, 2], a 16-32
    cell layer, K in {8, 12, 16} (one quarter layer nodes), 1-8 right-hand
    sides, tol 1e-6."""
    shape = grids[int(rng.integers(len(grids)))]
    N = shape[0]
    d = len(shape)
    width = int(rng.integers(16, 33))
    ppw = float(rng.uniform(6, 12))
    K = int(rng.choice([8, 12, 16]))
    Mt = K // 4
    nrhs = int(rng.integers(1, max_rhs + 1))
    nb = int(rng.integers(3, 11))
    raw = bumps(rng, shape, nb, lambda r: r.uniform(0.2, 1.0), lambda r: r.uniform(0.03, 0.1),
                width)
    raw = 1.0 + (raw - raw.min()) / max(raw.max() - raw.min(), 1e-30)
    c, zeta = finish_medium(raw, width, DEFAULT_ZETA_MAX)
    omega = omega_for_ppw(float(c.min()), N, ppw)
    f = point_sources(rng, shape, width, nrhs)
    return Problem(f"serve-{d}d-{N}", shape, c, zeta, None, omega, 1.0, K - Mt, Mt, f, 40,
                   1e-6, 1, width, meta=dict(ppw=ppw, width=width))


SHARED_MEDIA_GRIDS = [(256, 256), (512, 512), (1024, 1024), (64, 64, 64), (128, 128, 128)]


def shared_media_pool(n_media: int, seed: int = 16179, grids=SHARED_MEDIA_GRIDS) -> list:
    """A pool of media for a stream of requests that share them (many source
    positions on a few media): medium k is the serving recipe's medium drawn
    with seed [seed, k] over the given grids, with its own frequency, layer
    and K."""
    return [serving_request(np.random.Generator(np.random.PCG64([seed, k])), grids, max_rhs=1)
            for k in range(n_media)]


def shared_media_request(rng, pool, max_rhs: int = 4) -> Problem:
    """One request on a medium drawn uniformly from the pool: the medium's
    grid, c, zeta, omega and K, with 1..max_rhs new point sources."""
    base = pool[int(rng.integers(len(pool)))]
    nrhs = int(rng.integers(1, max_rhs + 1))
    f = point_sources(rng, base.shape, base.meta["width"], nrhs)
    return Problem(base.name + "-shared", base.shape, base.c, base.zeta, None, base.omega, 1.0,
                   base.M, base.Mt, f, base.restart, base.tol, base.precision, base.meta["width"],
                   meta=dict(base.meta))


def example1(N: int = 2048, *, ppw: float = 12.0, delta: float = 1.0, eta: float = 1.0 / 800,
             a: float = 20.0, M: int = 8, restart: int = 10) -> Problem:
    """The paper's Example 1 (Section 5.1): periodic unit square, circular
    inclusion c = c_o + delta H_eta(0.05 - |x|) with c_o = 1 (Eqn. WS),
    constant damping a, plane-wave source exp(i omega x_1 / c_o) along the
    x axis (Eqn. Source), omega from PPW = 2 pi c_o N / (L omega), M real
    nodes and no absorbing layer, GMRES(restart).  The symbol uses the
    operator's damping (a_node = a, alpha = 0 for the medium)."""
    shape = (N, N)
    X = coords(shape)
    r = np.sqrt(X[0] ** 2 + X[1] ** 2)
    c = np.broadcast_to(1.0 + delta * smooth_heaviside(0.05 - r, eta), shape).copy()
    omega = 2.0 * np.pi * 1.0 * N / ppw
    f = np.exp(1j * omega * np.broadcast_to(X[1], shape))[None].astype(np.complex128)
    return Problem(f"example1-{N}-ppw{ppw:g}-delta{delta:g}-a{a:g}-M{M}", shape, c,
                   np.zeros(shape), np.full(shape, float(a)), omega, 1.0, M, 0, f, restart,
                   1e-14, 0, 0, meta={"a_node": float(a), "alpha": 0.0, "eta": eta,
                                      "delta": delta, "ppw": ppw})


def random_field(rng, shape, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian test vector(s) with i.i.d. N(0,1) parts."""
    s = tuple(shape) if nrhs is None else (nrhs,) + tuple(shape)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


def small_problem(shape, seed: int, *, M: int = 4, Mt: int = 2, width: int = 2,
                  contrast: float = 0.5, ppw: float = 6.0, zeta_max: float = DEFAULT_ZETA_MAX,
                  a_const: float | None = None, damping: tuple | None = None) -> Problem:
    """A small smooth random medium for parity tests at any (ragged) shape:
    a few bumps of relative height `contrast`, a `width`-cell layer.
    damping = (lo, hi): a(x) = omega (lo + (hi - lo) b(x)), b an independent
    bump field scaled to [0, 1] (damping that does not follow c)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(shape)
    X = coords(shape)
    raw = np.zeros(shape)
    for _ in range(3):
        ctr = rng.uniform(-0.2, 0.2, size=len(shape))
        s = rng.uniform(0.08, 0.2)
        d2 = sum((X[ax] - ctr[ax]) ** 2 for ax in range(len(shape)))
        raw = raw + rng.uniform(0.3, 1.0) * np.exp(-d2 / (2 * s * s))
    raw = 1.0 + contrast * raw / max(raw.max(), 1e-30)
    if width > 0:
        c, zeta = finish_medium(raw, width, zeta_max, taper_cells=2)
    else:
        c, zeta = raw, np.zeros(shape)
    omega = omega_for_ppw(float(c.min()), min(shape), ppw)
    a = None if a_const is None else np.full(shape, float(a_const))
    if damping is not None:
        b = damping_field(rng, shape)
        a = omega * (damping[0] + (damping[1] - damping[0]) * b)
    f = random_field(rng, shape, 1)
    return Problem(f"small-{'x'.join(map(str, shape))}", shape, c, zeta, a, omega, 1.0, M, Mt,
                   f, 30, 1e-6, 0, width)


def damping_field(rng, shape, n_bumps: int = 4) -> np.ndarray:
    """An independent smooth field in [0, 1]: Gaussian bumps (sigma
    U[0.08, 0.25], amplitude U[0.3, 1]) at uniform centres, min-max scaled."""
    X = coords(shape)
    b = np.zeros(shape)
    for _ in range(n_bumps):
        ctr = rng.uniform(-0.4, 0.4, size=len(shape))
        s = rng.uniform(0.08, 0.25)
        d2 = sum((X[ax] - ctr[ax]) ** 2 for ax in range(len(shape)))
        b = b + rng.uniform(0.3, 1.0) * np.exp(-d2 / (2 * s * s))
    return (b - b.min()) / max(b.max() - b.min(), 1e-30)


def damping_problem(N: int = 1024, seed: int = 16179, *, Ma: int = 3,
                    damping: tuple = (0.02, 0.2), width: int = 32, ppw: float = 8.0,
                    M: int = 12, Mt: int = 4, nrhs: int = 1) -> Problem:
    """The 2D bumps + gradient medium of the 1024^2 workload at side N, with a
    damping field a(x) = omega (lo + (hi - lo) b(x)) that does not follow c
    (b: damping_field from the same seeded stream after c and f), for the
    bivariate (c, a) interpolation; FGMRES(40), complex64 preconditioner."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (N, N)
    raw = bumps(rng, shape, 20, lambda r: r.uniform(0, 1), lambda r: r.uniform(0.02, 0.1),
                width)
    X = coords(shape)
    raw = raw + 0.5 * (X[1] + 0.5)
    raw = 1.0 + (raw - raw.min()) / (raw.max() - raw.min())
    c, zeta = finish_medium(raw, width, DEFAULT_ZETA_MAX)
    omega = omega_for_ppw(float(c.min()), N, ppw)
    f = point_sources(rng, shape, width, nrhs)
    a = omega * (damping[0] + (damping[1] - damping[0]) * damping_field(rng, shape, 8))
    return Problem(f"2d-{N}-bumps20-grad-damping-Ma{Ma}", shape, c, zeta, a, omega, 1.0, M, Mt,
                   f, 40, 1e-6, 1, width, meta=dict(Ma=Ma, damping=damping))
