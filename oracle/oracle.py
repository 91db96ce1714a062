"""Python face of the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``liboracle.so`` (built from
``lgf_oracle.c`` with gcc + OpenMP) through ctypes and wraps it with numpy.
Nothing here touches the CUDA library, and the CUDA library never calls this.

Functions (each cites the passage of Liska & Colonius, arXiv:1604.01814, that
it follows; the C source documents the numerical method):
  ive_all            e^{-z} I_k(z), k = 0..nmax                App. A, Eq. lgf_intfac
  lgf_quad           G_L(n) by quadrature of the Bessel form    App. A, Eq. lgf_lap
  lgf_asym           far-field expansion of G_L                  Sec. 2.2 / App. A footnote
  lgf_table          G_L over sorted offsets up to R             App. A (look-up table)
  poisson_direct     u = dx^2 sum_m G_L(n-m) f(m)                Sec. 2.2, Eq. dpoisson_conv
  poisson_direct_multi  the same for several fields on one source set
  intfactor_weights  e^{-2a} I_n(2a), n = 0..nmax                App. A, Eq. lgf_intfac
  intfactor_box      u = E(alpha) f on a dense box (untruncated) Sec. 2.3 footnote
  lgf_r              R(alpha)(n) = int_0^alpha G_E(t)(n) dt      App. A (partition of G_K)
  gk_quad, gk_table  G_K(alpha) = G_L + R(alpha)                 App. A, Eq. lgf_iflap
  kinv_direct        u = dx^2 sum_m G_K(alpha)(n-m) f(m)         Sec. 2.2 (action of K^{-1})
  curl_box           C: faces -> edges (staggered curl)          Sec. 2.1 (operator list)
  curl_adj_box       C^dagger: edges -> faces (adjoint of C)     Sec. 2.1
  grad_box, div_box  G: cells -> faces, Dbar = -G^dagger          Sec. 2.1 (pins only)
  velocity_refresh   w = C u, s = L^{-1} w, u = -C^dagger s      Sec. 4.1, Eq. vel_refresh
  phi3               three-point kernel phi(r) (reading: Roma-Peskin-Berger)  Sec. 2.1
  ib_spread          (R g)^k(n) = sum_i g^k(i) delta_dx(x_F^k(n) - X_i)       Sec. 2.1 (operator R)
  ib_interp          (I v)^k(i) = dx^3 sum_n v^k(n) delta_dx(x_F^k(n) - X_i)  Sec. 2.1 (operator I)
  nested_projection_stage  ip -> f -> pc -> vc of one IF-HERK stage   Sec. 3.1, Eq. nested_proj
  force_schur        C = I H S I^dagger, S = I - G L_C^{-1} Dbar (dense)  Sec. 3.1, Eq. force_schur
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O3 -fopenmp; no contraction of a*b+c into one rounding, so the
    arithmetic is the same plain IEEE evaluation on every host).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_ive_all.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
            L.orc_gk15_poly.argtypes = [ctypes.c_int, _dp, _dp]
            L.orc_lgf_quad.argtypes = [ctypes.c_int] * 3
            L.orc_lgf_quad.restype = ctypes.c_double
            L.orc_lgf_asym.argtypes = [ctypes.c_int] * 4
            L.orc_lgf_asym.restype = ctypes.c_double
            L.orc_table_index.argtypes = [ctypes.c_int] * 3
            L.orc_table_index.restype = ctypes.c_int64
            L.orc_table_size.argtypes = [ctypes.c_int]
            L.orc_table_size.restype = ctypes.c_int64
            L.orc_lgf_table.argtypes = [ctypes.c_int, _dp]
            L.orc_lgf.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_lgf.restype = ctypes.c_double
            L.orc_poisson_direct.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_int64, _ip,
                                             ctypes.c_double, _dp, ctypes.c_int, _dp]
            L.orc_poisson_direct_multi.argtypes = [ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int, _dp, ctypes.c_int64,
                                                   _ip, ctypes.c_double, _dp, ctypes.c_int, _dp]
            L.orc_intfactor_weights.argtypes = [ctypes.c_double, ctypes.c_int, _dp]
            L.orc_intfactor_box.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_lgf_r.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_lgf_r.restype = ctypes.c_double
            L.orc_gk_quad.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_gk_quad.restype = ctypes.c_double
            L.orc_r_table.argtypes = [ctypes.c_double, ctypes.c_int, _dp]
            _lib = L
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def ive_all(nmax: int, z: float) -> np.ndarray:
    out = np.empty(nmax + 1)
    if lib().orc_ive_all(int(nmax), float(z), _p(out)) != 0:
        raise ValueError("bad arguments")
    return out


def gk15_poly(k: int):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_gk15_poly(int(k), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def lgf_quad(n1: int, n2: int, n3: int) -> float:
    return float(lib().orc_lgf_quad(int(n1), int(n2), int(n3)))


def lgf_asym(n1: int, n2: int, n3: int, order: int = 7) -> float:
    return float(lib().orc_lgf_asym(int(n1), int(n2), int(n3), int(order)))


def table_index(a: int, b: int, c: int) -> int:
    return int(lib().orc_table_index(a, b, c))


_table_cache: dict[int, np.ndarray] = {}


def lgf_table(R: int) -> np.ndarray:
    """G_L over sorted offsets a >= b >= c >= 0, a <= R (cached per process)."""
    R = int(R)
    if R not in _table_cache:
        n = int(lib().orc_table_size(R))
        out = np.empty(n)
        if lib().orc_lgf_table(R, _p(out)) != 0:
            raise RuntimeError("orc_lgf_table failed")
        _table_cache[R] = out
    return _table_cache[R]


def lgf(n, R: int = 32) -> np.ndarray:
    """G_L at integer offsets n (shape [..., 3]); table up to R, expansion beyond."""
    n = np.asarray(n, dtype=np.int64).reshape(-1, 3)
    tab = lgf_table(R)
    L = lib()
    out = np.array([L.orc_lgf(_p(tab), R, int(a), int(b), int(c)) for a, b, c in n])
    return out


def poisson_direct(b: int, src_coords, f, tgt_pts, dx: float = 1.0, R: int = 32) -> np.ndarray:
    """u(t) = dx^2 sum_{m in src blocks} G_L(t - m) f(m) at lattice points tgt_pts [n][3].

    f: [nsrc][b^3] (x fastest inside a block), float64."""
    src = np.ascontiguousarray(src_coords, dtype=np.int32).reshape(-1, 3)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(src.shape[0], b ** 3)
    tp = np.ascontiguousarray(tgt_pts, dtype=np.int32).reshape(-1, 3)
    tab = lgf_table(R)
    out = np.empty(tp.shape[0])
    rc = lib().orc_poisson_direct(int(b), src.shape[0], _p(src, _ip), _p(f), tp.shape[0], _p(tp, _ip),
                                  float(dx), _p(tab), int(R), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_poisson_direct failed ({rc})")
    return out


def poisson_direct_multi(b: int, src_coords, f, tgt_pts, dx: float = 1.0, R: int = 32) -> np.ndarray:
    """poisson_direct for several fields on one source set: f [nf][nsrc][b^3]
    -> [nf][ntgt] (one G_L evaluation per pair serves every field)."""
    src = np.ascontiguousarray(src_coords, dtype=np.int32).reshape(-1, 3)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, src.shape[0], b ** 3)
    tp = np.ascontiguousarray(tgt_pts, dtype=np.int32).reshape(-1, 3)
    tab = lgf_table(R)
    out = np.empty((f.shape[0], tp.shape[0]))
    rc = lib().orc_poisson_direct_multi(int(b), src.shape[0], _p(src, _ip), f.shape[0], _p(f), tp.shape[0],
                                        _p(tp, _ip), float(dx), _p(tab), int(R), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_poisson_direct_multi failed ({rc})")
    return out


def intfactor_weights(alpha: float, nmax: int) -> np.ndarray:
    out = np.empty(nmax + 1)
    if lib().orc_intfactor_weights(float(alpha), int(nmax), _p(out)) != 0:
        raise ValueError("bad arguments")
    return out


def intfactor_box(alpha: float, f_box: np.ndarray) -> np.ndarray:
    """u = E(alpha) f on a dense box f_box[z, y, x]; every offset inside the box kept."""
    f = np.ascontiguousarray(f_box, dtype=np.float64)
    nz, ny, nx = f.shape
    u = np.empty_like(f)
    if lib().orc_intfactor_box(float(alpha), nx, ny, nz, _p(f), _p(u)) != 0:
        raise RuntimeError("orc_intfactor_box failed")
    return u


# ----------------------------------------------------------------------------
# Block-set helpers (pure data movement between block layout and dense boxes).
# ----------------------------------------------------------------------------
def blocks_to_box(b: int, coords, vals, lo=None, shape=None):
    """Scatter block-layout values [nblk][b^3] into a dense box [z, y, x]."""
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    if lo is None:
        lo = coords.min(axis=0)
    if shape is None:
        hi = coords.max(axis=0) + 1
        shape = tuple(int(v) for v in ((hi - lo) * b)[::-1])
    box = np.zeros(shape)
    v = np.asarray(vals, dtype=np.float64).reshape(-1, b, b, b)
    for i, (cx, cy, cz) in enumerate(coords - lo):
        box[cz * b:(cz + 1) * b, cy * b:(cy + 1) * b, cx * b:(cx + 1) * b] = v[i]
    return box, lo


def box_to_blocks(b: int, coords, box, lo):
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    out = np.empty((coords.shape[0], b, b, b))
    for i, (cx, cy, cz) in enumerate(coords - np.asarray(lo)):
        out[i] = box[cz * b:(cz + 1) * b, cy * b:(cy + 1) * b, cx * b:(cx + 1) * b]
    return out.reshape(coords.shape[0], b ** 3)


def intfactor_blocks(alpha: float, b: int, src_coords, f, tgt_coords) -> np.ndarray:
    """u = E(alpha) f restricted to the target blocks; f is zero outside src blocks."""
    src = np.asarray(src_coords).reshape(-1, 3)
    tgt = np.asarray(tgt_coords).reshape(-1, 3)
    allc = np.concatenate([src, tgt])
    lo = allc.min(axis=0)
    hi = allc.max(axis=0) + 1
    shape = tuple(int(v) for v in ((hi - lo) * b)[::-1])
    box, _ = blocks_to_box(b, src, f, lo, shape)
    u = intfactor_box(alpha, box)
    return box_to_blocks(b, tgt, u, lo)


def block_points(b: int, coords) -> np.ndarray:
    """All lattice points of the blocks, in block layout order: [nblk*b^3][3] (x, y, z)."""
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    r = np.arange(b)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    loc = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return (coords[:, None, :] * b + loc[None, :, :]).reshape(-1, 3)


def lgf_r(alpha: float, n1: int, n2: int, n3: int) -> float:
    """R(alpha)(n) = int_0^alpha prod_i e^{-2t} I_{|n_i|}(2t) dt (App. A)."""
    return float(lib().orc_lgf_r(float(alpha), int(n1), int(n2), int(n3)))


def gk_quad(alpha: float, n1: int, n2: int, n3: int) -> float:
    """G_K(alpha)(n) = G_L(n) + R(alpha)(n) (App. A, Eq. lgf_iflap)."""
    return float(lib().orc_gk_quad(float(alpha), int(n1), int(n2), int(n3)))


_gk_cache: dict = {}


def gk_table(alpha: float, R: int) -> np.ndarray:
    """G_K(alpha) over sorted offsets a >= b >= c >= 0, a <= R (cached)."""
    key = (float(alpha), int(R))
    if key not in _gk_cache:
        r = np.empty(int(lib().orc_table_size(int(R))))
        if lib().orc_r_table(float(alpha), int(R), _p(r)) != 0:
            raise RuntimeError("orc_r_table failed")
        _gk_cache[key] = lgf_table(R) + r
    return _gk_cache[key]


def gk(n, alpha: float, R: int = 32) -> np.ndarray:
    """G_K(alpha) at integer offsets n [..., 3]: table up to R, the G_L
    expansion beyond (R(alpha) is below 1e-9 |G_L(0)| there for alpha <= 1,
    App. A footnote; tests check the shell)."""
    n = np.asarray(n, dtype=np.int64).reshape(-1, 3)
    tab = gk_table(alpha, R)
    L = lib()
    return np.array([L.orc_lgf(_p(tab), int(R), int(a), int(b), int(c)) for a, b, c in n])


def kinv_direct(alpha: float, b: int, src_coords, f, tgt_pts, dx: float = 1.0, R: int = 32) -> np.ndarray:
    """u(t) = dx^2 sum_{m in src blocks} G_K(alpha)(t - m) f(m): the action of
    K(alpha)^{-1} = [E(-alpha) L]^{-1} (Sec. 2.2) by direct summation."""
    src = np.ascontiguousarray(src_coords, dtype=np.int32).reshape(-1, 3)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(src.shape[0], b ** 3)
    tp = np.ascontiguousarray(tgt_pts, dtype=np.int32).reshape(-1, 3)
    tab = gk_table(alpha, R)
    out = np.empty(tp.shape[0])
    rc = lib().orc_poisson_direct(int(b), src.shape[0], _p(src, _ip), _p(f), tp.shape[0], _p(tp, _ip),
                                  float(dx), _p(tab), int(R), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_poisson_direct failed ({rc})")
    return out


# ----------------------------------------------------------------------------
# Staggered-grid operators (Sec. 2.1) on dense boxes [3][z][y][x], zero outside.
# Cell n of the lattice holds face k at (n + (1 - e_k)/2) dx and edge k at
# (n + e_k/2) dx; a vector field stores component k of cell n at [k][z][y][x].
# The paper lists C: faces -> edges and its adjoint C^dagger but prints no
# stencil; these are the standard second-order finite-volume (MAC) ones, and
# the tests pin them to the paper's mimetic identity L_F = -G G^dagger - C^dagger C.
# ----------------------------------------------------------------------------
_AX = {0: 2, 1: 1, 2: 0}   # lattice axis k -> array axis of [z][y][x]


def _shift(a: np.ndarray, k: int, d: int) -> np.ndarray:
    """b(n) = a(n + d e_k) on the same box (the last three array axes are z, y, x),
    zero where n + d e_k leaves it."""
    out = np.zeros_like(a)
    ax = a.ndim - 3 + _AX[k]
    n = a.shape[ax]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if d > 0:
        src[ax], dst[ax] = slice(d, n), slice(0, n - d)
    else:
        src[ax], dst[ax] = slice(0, n + d), slice(-d, n)
    out[tuple(dst)] = a[tuple(src)]
    return out


_EPS = ((0, 1, 2), (1, 2, 0), (2, 0, 1))   # (k, i, j) with eps_kij = +1


def curl_box(u: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """(C u)_k(n) = [u_j(n) - u_j(n - e_i)] - [u_i(n) - u_i(n - e_j)] / dx, (k,i,j) cyclic:
    the circulation of the face velocities around edge k (backward differences)."""
    w = np.empty_like(u)
    for k, i, j in _EPS:
        w[k] = ((u[j] - _shift(u[j], i, -1)) - (u[i] - _shift(u[i], j, -1))) / dx
    return w


def curl_adj_box(w: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """(C^dagger w)_k(m) = [w_i(m) - w_i(m + e_j)] - [w_j(m) - w_j(m + e_i)] / dx: the adjoint
    of curl_box under sum_n a(n) b(n) (forward differences)."""
    u = np.empty_like(w)
    for k, i, j in _EPS:
        u[k] = ((w[i] - _shift(w[i], j, +1)) - (w[j] - _shift(w[j], i, +1))) / dx
    return u


def grad_box(q: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """(G q)_k(n) = [q(n) - q(n - e_k)] / dx: cells -> faces."""
    return np.stack([(q - _shift(q, k, -1)) / dx for k in range(3)])


def div_box(u: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """(Dbar u)(n) = sum_k [u_k(n + e_k) - u_k(n)] / dx = -(G^dagger u)(n): faces -> cells."""
    return sum((_shift(u[k], k, +1) - u[k]) / dx for k in range(3))


def lap_box(a: np.ndarray, dx: float = 1.0) -> np.ndarray:
    """7-point Laplacian of each component (the scalar L of Sec. 2.2 applied componentwise)."""
    out = -6.0 * a
    for k in range(3):
        out = out + _shift(a, k, 1) + _shift(a, k, -1)
    return out / dx ** 2


def _vec_to_box(b: int, coords, v, lo, shape):
    v = np.asarray(v, dtype=np.float64).reshape(3, -1)
    return np.stack([blocks_to_box(b, coords, v[k], lo, shape)[0] for k in range(3)])


def _vec_from_box(b: int, coords, box, lo):
    return np.stack([box_to_blocks(b, coords, box[k], lo) for k in range(3)])


def grown_forward(coords) -> np.ndarray:
    """The block set with every block's +x, +y and +z neighbours added (sorted)."""
    c = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    out = {tuple(r) for r in c}
    for e in np.eye(3, dtype=np.int64):
        out |= {tuple(r) for r in c + e}
    return np.array(sorted(out), dtype=np.int32)


def velocity_refresh(b: int, src_coords, u, tgt_coords, dx: float = 1.0, R: int = 64) -> np.ndarray:
    """Velocity refresh of Eq. vel_refresh on block sets: w = C u on the source blocks
    (u zero outside them), s = L^{-1} w = dx^2 G_L * w (each edge component a scalar
    convolution) on the target blocks and their forward neighbours, u_new = -C^dagger s
    on the target blocks.  The minus sign is the reading of the printed composition that
    returns a divergence-free u unchanged (with L_F = -G G^dagger - C^dagger C, Sec. 2.1).
    u: [3][nsrc][b^3]; returns [3][ntgt][b^3]."""
    src = np.asarray(src_coords, dtype=np.int64).reshape(-1, 3)
    tgt = np.asarray(tgt_coords, dtype=np.int64).reshape(-1, 3)
    tg = grown_forward(tgt).astype(np.int64)
    allc = np.concatenate([src, tg])
    lo = allc.min(axis=0)
    hi = allc.max(axis=0) + 1
    shape = tuple(int(v) for v in ((hi - lo) * b)[::-1])
    ubox = _vec_to_box(b, src, u, lo, shape)
    w = _vec_from_box(b, src, curl_box(ubox, dx), lo)           # C u, kept on the source blocks
    pts = block_points(b, tg)
    s = np.stack([poisson_direct(b, src, w[k], pts, dx=dx, R=R).reshape(tg.shape[0], b ** 3)
                  for k in range(3)])
    sbox = _vec_to_box(b, tg, s, lo, shape)
    return -_vec_from_box(b, tgt, curl_adj_box(sbox, dx), lo)


# ----------------------------------------------------------------------------
# Immersed-boundary regularisation R and interpolation I (Sec. 2.1): face k of
# cell n sits at x_F^k(n) = (n + (1 - e_k)/2) dx; delta_h(x) = h^-3 prod_d
# phi(x_d / h).  Marker positions X are given in units of dx.  Plain loops over
# markers and the 4 x 4 x 4 lattice points around each (phi vanishes beyond
# |r| = 3/2, so the extra ring only adds zeros).
# ----------------------------------------------------------------------------
def phi3(r):
    """phi(r) = (1 + sqrt(1 - 3 r^2)) / 3 for |r| <= 1/2,
    (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6 for 1/2 <= |r| <= 3/2, 0 beyond."""
    a = abs(float(r))
    if a <= 0.5:
        return (1.0 + math.sqrt(1.0 - 3.0 * a * a)) / 3.0
    if a <= 1.5:
        return (5.0 - 3.0 * a - math.sqrt(max(0.0, 1.0 - 3.0 * (1.0 - a) ** 2))) / 6.0
    return 0.0


def _block_lookup(b: int, coords):
    c = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    return {tuple(v): i for i, v in enumerate(c.tolist())}


def _ib_points(X, k):
    """Lattice cells n whose face k may lie within 3/2 of X (per axis), with weights."""
    o = [0.5, 0.5, 0.5]
    o[k] = 0.0
    base = [int(math.floor(X[d] - o[d])) - 1 for d in range(3)]
    for dz in range(4):
        for dy in range(4):
            for dx_ in range(4):
                n = (base[0] + dx_, base[1] + dy, base[2] + dz)
                w = phi3(n[0] + o[0] - X[0]) * phi3(n[1] + o[1] - X[1]) * phi3(n[2] + o[2] - X[2])
                if w != 0.0:
                    yield n, w


def ib_spread(b: int, coords, X, g, dx: float = 1.0) -> np.ndarray:
    """f = R g on the face lattices of the blocks: g [nrhs][3][nm] -> [nrhs][3][nblk][b^3].
    Points outside the block set are dropped."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    g = np.asarray(g, dtype=np.float64)
    # no markers: one right-hand side of nothing to spread (an empty array has no size to infer it from)
    g = g.reshape(-1, 3, X.shape[0]) if X.shape[0] else np.zeros((1, 3, 0))
    lut = _block_lookup(b, coords)
    out = np.zeros((g.shape[0], 3, len(lut), b ** 3))
    for i in range(X.shape[0]):
        for k in range(3):
            for n, w in _ib_points(X[i], k):
                blk = lut.get((n[0] // b, n[1] // b, n[2] // b))
                if blk is None:
                    continue
                loc = ((n[2] % b) * b + n[1] % b) * b + n[0] % b
                out[:, k, blk, loc] += w * g[:, k, i] / dx ** 3
    return out


def ib_interp(b: int, coords, X, v) -> np.ndarray:
    """U = I v at the markers: v [nrhs][3][nblk][b^3] -> [nrhs][3][nm]
    (dx^3 delta_dx = prod phi, so dx drops out).  Absent blocks read as zero."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    lut = _block_lookup(b, coords)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3, len(lut), b ** 3)
    out = np.zeros((v.shape[0], 3, X.shape[0]))
    for i in range(X.shape[0]):
        for k in range(3):
            for n, w in _ib_points(X[i], k):
                blk = lut.get((n[0] // b, n[1] // b, n[2] // b))
                if blk is None:
                    continue
                loc = ((n[2] % b) * b + n[1] % b) * b + n[0] % b
                out[:, k, i] += w * v[:, k, blk, loc]
    return out



# ----------------------------------------------------------------------------
# One IF-HERK stage's linear solve by the nested projection of Sec. 3.1
# (Eq. nested_proj), on one flow block set D with sources and results
# truncated to D (Table 1's truncation, reading 4).  The Poisson problems'
# targets are D and its -x, -y, -z neighbour blocks (the cells that the
# gradient on the faces of D reads).  Fields on D: r, u faces [3][nD][b^3];
# cells [nD][b^3].  Markers X (stage i) and X_prev (stage i-1) in units of dx,
# marker vectors [3][nm].  The force Schur complement's inverse is given as
# factors: f_hat = W2 (W1 rhs), W2 = W1^T when omitted (the Cholesky form of
# Sec. 3.2, C^-1 = W^T W).  Each step is a module function so that the
# mutation tests can plant a mistake in one of them (`ops`).
# ----------------------------------------------------------------------------
def grown_backward(coords) -> np.ndarray:
    """D followed by the blocks at -x, -y, -z of D that are not in D (sorted)."""
    c = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    have = {tuple(r) for r in c}
    extra = set()
    for e in np.eye(3, dtype=np.int64):
        extra |= {tuple(r) for r in c - e} - have
    ext = np.array(sorted(extra), dtype=np.int64).reshape(-1, 3)
    return np.concatenate([c, ext]).astype(np.int32)


class _StageGeom:
    def __init__(self, b, D):
        self.b = b
        self.D = np.asarray(D, dtype=np.int64).reshape(-1, 3)
        self.Dm = grown_backward(self.D).astype(np.int64)
        self.lo = self.Dm.min(axis=0)
        hi = self.Dm.max(axis=0) + 1
        self.shape = tuple(int(v) for v in ((hi - self.lo) * b)[::-1])

    def faces_box(self, v):
        return _vec_to_box(self.b, self.D, v, self.lo, self.shape)

    def faces_on_D(self, box):
        return _vec_from_box(self.b, self.D, box, self.lo)

    def cells_box(self, q, coords):
        return blocks_to_box(self.b, coords, q, self.lo, self.shape)[0]

    def cells_on(self, box, coords):
        return box_to_blocks(self.b, coords, box, self.lo)


def stage_lap_inv(g: _StageGeom, q, dx, R):
    """L_C^{-1} q = dx^2 G_L * q (Sec. 2.2): sources on the cells of D, values
    on the cells of D and its backward neighbours."""
    return poisson_direct(g.b, g.D, q, block_points(g.b, g.Dm), dx=dx, R=R).reshape(g.Dm.shape[0], -1)


def stage_ip(g: _StageGeom, r, dx, R, ops):
    """Eq. nested_proj-ip: L_C d* = -G^dagger r, and -G^dagger = Dbar (Sec. 2.1)."""
    q = g.cells_on(ops.div_box(g.faces_box(r), dx), g.D)
    return ops.stage_lap_inv(g, q, dx, R)


def stage_f_rhs(g: _StageGeom, r, dstar, X, ub, alpha, dx, ops):
    """Right side of Eq. nested_proj-f: I^i H^i [r - G d*] - u_Gamma (printed
    H_C [r - G^dagger d*]; read as the face operators, see the readings)."""
    v = g.faces_on_D(g.faces_box(r) - ops.grad_box(g.cells_box(dstar, g.Dm), dx))
    w = np.stack([ops.intfactor_blocks(alpha, g.b, g.D, v[k], g.D) for k in range(3)])
    return ops.ib_interp(g.b, g.D, X, w[None])[0] - np.asarray(ub, dtype=np.float64).reshape(3, -1)


def stage_regularize(g: _StageGeom, X_prev, fhat, dx, ops):
    """(I^{i-1})^dagger f_hat = dx^3 R f_hat on the faces of D (I = dx^3 R^dagger, Sec. 2.1)."""
    return dx ** 3 * ops.ib_spread(g.b, g.D, X_prev, np.asarray(fhat).reshape(1, 3, -1), dx)[0]


def stage_pc(g: _StageGeom, dstar, gfaces, dx, R, ops):
    """Eq. nested_proj-pc: d_hat = d* + L_C^{-1} G^dagger (I^{i-1})^dagger f_hat,
    G^dagger = -Dbar."""
    q2 = -g.cells_on(ops.div_box(g.faces_box(gfaces), dx), g.D)
    return dstar + ops.stage_lap_inv(g, q2, dx, R)


def stage_vc(g: _StageGeom, r, dhat, gfaces, alpha, dx, ops):
    """Eq. nested_proj-vc: u = H^i [r - G d_hat - (I^{i-1})^dagger f_hat]."""
    v = g.faces_on_D(g.faces_box(r) - ops.grad_box(g.cells_box(dhat, g.Dm), dx) - g.faces_box(gfaces))
    return np.stack([ops.intfactor_blocks(alpha, g.b, g.D, v[k], g.D) for k in range(3)])


def nested_projection_stage(b: int, D, r, X_prev, X, ub, W1, W2=None, alpha: float = 0.0, dx: float = 1.0,
                            R: int = 64, ops=None):
    """Eq. nested_proj for one stage: ip -> f -> pc -> vc.  Returns (u [3][nD][b^3],
    d_hat on the cells of D [nD][b^3], f_hat [3][nm])."""
    import sys
    ops = ops if ops is not None else sys.modules[__name__]
    g = _StageGeom(b, D)
    r = np.asarray(r, dtype=np.float64).reshape(3, g.D.shape[0], b ** 3)
    dstar = ops.stage_ip(g, r, dx, R, ops)
    rhs = ops.stage_f_rhs(g, r, dstar, X, ub, alpha, dx, ops)
    W1 = np.asarray(W1, dtype=np.float64)
    W2 = W1.T if W2 is None else np.asarray(W2, dtype=np.float64)
    fhat = (W2 @ (W1 @ rhs.reshape(-1))).reshape(3, -1)
    gf = ops.stage_regularize(g, X_prev, fhat, dx, ops)
    dhat = ops.stage_pc(g, dstar, gf, dx, R, ops)
    u = ops.stage_vc(g, r, dhat, gf, alpha, dx, ops)
    return u, dhat[:g.D.shape[0]], fhat


def force_schur(b: int, D, X_prev, X, alpha: float = 0.0, dx: float = 1.0, R: int = 64) -> np.ndarray:
    """The force Schur complement C^i as a dense matrix, column by column, from
    its form I^i H^i S (I^{i-1})^dagger with S = I - G L_C^{-1} Dbar (Sec. 3.1;
    printed L_F^{-1}, read as the cell Laplacian), on the truncation of
    nested_projection_stage.  Rows and columns in the [3][nm] order."""
    g = _StageGeom(b, D)
    nm = np.asarray(X).reshape(-1, 3).shape[0]
    C = np.zeros((3 * nm, 3 * nm))
    for j in range(3 * nm):
        e = np.zeros(3 * nm)
        e[j] = 1.0
        s = stage_regularize(g, X_prev, e.reshape(3, nm), dx, sys_mod())
        q = g.cells_on(div_box(g.faces_box(s), dx), g.D)          # Dbar s
        p = stage_lap_inv(g, q, dx, R)                              # L_C^{-1} Dbar s
        v = g.faces_on_D(g.faces_box(s) - grad_box(g.cells_box(p, g.Dm), dx))
        w = np.stack([intfactor_blocks(alpha, b, g.D, v[k], g.D) for k in range(3)])
        C[:, j] = ib_interp(b, g.D, X, w[None])[0].reshape(-1)
    return C


def sys_mod():
    import sys
    return sys.modules[__name__]
