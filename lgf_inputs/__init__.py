"""Seeded synthetic inputs for the LGF Poisson and integrating-factor applies.

This module is shared by the tests, the benchmark and the smoke check.  It holds
no arithmetic of the method itself (no Green's function, no Bessel factor, no
convolution): it only draws block sets and source fields with the shapes of the
workloads of Liska & Colonius (arXiv:1604.01814) -- a dense box, a sphere with
its wake (Sec. 5.3) and low-aspect-ratio flat plates (Sec. 5.2) -- from
``numpy.random.default_rng(seed)``.

Layout conventions (the library's): a block set is an int32 array [nblocks][3]
of block coordinates (x, y, z); block B with edge b covers lattice points
b*B + [0, b)^3; a field on a block set is [nblocks][b^3] with x fastest inside a
block.  Multi-field arrays are [nrhs][ncomp][nblocks][b^3].

Immersed-boundary sources are spread from Lagrangian markers with a 3-point
regularised delta function.  The paper uses the smoothed kernel of Yang et al.
(2009), whose formula it does not print; these inputs use the three-point kernel
of Roma, Peskin & Berger (1999) instead, which only changes the shape of the
synthetic source (both sides of every parity test read the same arrays).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# Containers
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One apply: sources on ``src`` blocks, results wanted on ``tgt`` blocks."""
    name: str
    b: int
    src: np.ndarray            # [nsrc][3] int32
    tgt: np.ndarray            # [ntgt][3] int32
    f: np.ndarray              # [nrhs][ncomp][nsrc][b^3] float64
    alphas: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def nrhs(self):
        return self.f.shape[0]

    @property
    def ncomp(self):
        return self.f.shape[1]

    def target_points(self) -> int:
        return int(self.tgt.shape[0]) * self.b ** 3 * self.nrhs * self.ncomp


# ----------------------------------------------------------------------------
# Block-set helpers
# ----------------------------------------------------------------------------
def box_blocks(nbx: int, nby: int, nbz: int, origin=(0, 0, 0)) -> np.ndarray:
    """All blocks of an nbx x nby x nbz box, x fastest."""
    z, y, x = np.meshgrid(np.arange(nbz), np.arange(nby), np.arange(nbx), indexing="ij")
    c = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1) + np.asarray(origin)
    return c.astype(np.int32)


def block_point_coords(b: int, coords: np.ndarray) -> np.ndarray:
    """Lattice coordinates of every point of the blocks, [nblk, b, b, b, 3] (x, y, z)."""
    r = np.arange(b)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    loc = np.stack([x, y, z], axis=-1)
    return coords[:, None, None, None, :].astype(np.int64) * b + loc[None]


def random_blockset(rng, nblocks: int, extent, origin=(0, 0, 0)) -> np.ndarray:
    """``nblocks`` distinct blocks drawn uniformly from a box of ``extent`` blocks."""
    ex = np.asarray(extent)
    total = int(np.prod(ex))
    if nblocks > total:
        raise ValueError("more blocks than the box holds")
    idx = np.sort(rng.choice(total, size=nblocks, replace=False))
    x = idx % ex[0]
    y = (idx // ex[0]) % ex[1]
    z = idx // (ex[0] * ex[1])
    return (np.stack([x, y, z], axis=1) + np.asarray(origin)).astype(np.int32)


# ----------------------------------------------------------------------------
# Regularised delta and Lagrangian markers
# ----------------------------------------------------------------------------
def delta3(r: np.ndarray) -> np.ndarray:
    """Three-point kernel phi(r) of Roma, Peskin & Berger (support |r| < 3/2)."""
    a = np.abs(r)
    out = np.zeros_like(a, dtype=np.float64)
    m1 = a <= 0.5
    out[m1] = (1.0 + np.sqrt(1.0 - 3.0 * a[m1] ** 2)) / 3.0
    m2 = (a > 0.5) & (a <= 1.5)
    out[m2] = (5.0 - 3.0 * a[m2] - np.sqrt(np.maximum(0.0, 1.0 - 3.0 * (1.0 - a[m2]) ** 2))) / 6.0
    return out


def icosphere_markers(level: int) -> np.ndarray:
    """Unit-sphere markers at the face centroids of an icosahedron subdivided
    ``level - 1`` times (20 * 4^(level-1) markers), projected onto the sphere."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level - 1):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces)
    cen = V[F].mean(axis=1)
    return cen / np.linalg.norm(cen, axis=1, keepdims=True)


def plate_markers(chord: float, span: float, spacing: float, aoa_deg: float) -> np.ndarray:
    """Markers on a uniform grid over a flat plate (chord along x, span along z)
    pitched by ``aoa_deg`` about z, centred at the origin."""
    nc = max(2, int(round(chord / spacing)) + 1)
    ns = max(2, int(round(span / spacing)) + 1)
    s = (np.arange(nc) - (nc - 1) / 2.0) * (chord / (nc - 1))
    w = (np.arange(ns) - (ns - 1) / 2.0) * (span / (ns - 1))
    S, W = np.meshgrid(s, w, indexing="ij")
    a = math.radians(aoa_deg)
    x = S.ravel() * math.cos(a)
    y = -S.ravel() * math.sin(a)
    return np.stack([x, y, W.ravel()], axis=1)


def face_offset(k: int) -> np.ndarray:
    """Position of face-lattice component k inside cell n: n + (1 - e_k) / 2."""
    o = np.full(3, 0.5)
    o[k] = 0.0
    return o


def support_points(X: np.ndarray):
    """Yield (k, n [m][3], w [m], marker index [m]) for every face-lattice point
    n of component k that gets a non-zero 3-point weight from a marker."""
    off = np.arange(-2, 3)
    for k in range(3):
        P = X - face_offset(k)                       # lattice-index coordinates
        base = np.floor(P).astype(np.int64)
        for dz in off:
            for dy in off:
                for dx in off:
                    n = base + np.array([dx, dy, dz])
                    w = delta3(P[:, 0] - n[:, 0]) * delta3(P[:, 1] - n[:, 1]) * delta3(P[:, 2] - n[:, 2])
                    keep = np.nonzero(w != 0.0)[0]
                    if keep.size:
                        yield k, n[keep], w[keep], keep


def spread_to_blocks(b: int, coords: np.ndarray, X: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Spread marker forces F [nm][3] at positions X [nm][3] (cell units) onto
    the three face lattices, restricted to the given blocks: returns
    [3][nblk][b^3].  Points outside the block set are dropped."""
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    out = np.zeros((3, coords.shape[0], b ** 3))
    if coords.shape[0] == 0:
        return out
    lo = coords.min(axis=0)
    ext = coords.max(axis=0) - lo + 1
    lut = -np.ones(tuple(ext[::-1]), dtype=np.int64)          # [z][y][x] -> block index
    c = coords - lo
    lut[c[:, 2], c[:, 1], c[:, 0]] = np.arange(coords.shape[0])
    for k, n, w, mi in support_points(X):
        blk = np.floor_divide(n, b) - lo
        inside = np.all((blk >= 0) & (blk < ext), axis=1)
        idx = -np.ones(n.shape[0], dtype=np.int64)
        bi = blk[inside]
        idx[inside] = lut[bi[:, 2], bi[:, 1], bi[:, 0]]
        ok = idx >= 0
        loc = n[ok] - np.floor_divide(n[ok], b) * b
        lin = (loc[:, 2] * b + loc[:, 1]) * b + loc[:, 0]
        np.add.at(out[k], (idx[ok], lin), w[ok] * F[mi[ok], k])
    return out


def blocks_touched(b: int, X: np.ndarray) -> np.ndarray:
    """Blocks holding any face-lattice point that gets a non-zero weight from X."""
    parts = [np.floor_divide(n, b) for _, n, _, _ in support_points(X)]
    if not parts:
        return np.zeros((0, 3), dtype=np.int32)
    allb = np.concatenate(parts) + (1 << 20)
    key = np.unique((allb[:, 0] << 42) | (allb[:, 1] << 21) | allb[:, 2])   # sorted by (x, y, z)
    u = np.stack([key >> 42, (key >> 21) & ((1 << 21) - 1), key & ((1 << 21) - 1)], axis=1) - (1 << 20)
    return u.astype(np.int32).reshape(-1, 3)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
def uniform_box(b: int = 32, nb=(1, 1, 1), seed: int = 0, nrhs: int = 1, ncomp: int = 1) -> Problem:
    """Dense box of nb blocks, f i.i.d. uniform[-1, 1]."""
    rng = np.random.default_rng(seed)
    c = box_blocks(*nb)
    f = rng.uniform(-1.0, 1.0, size=(nrhs, ncomp, c.shape[0], b ** 3))
    return Problem("uniform_box", b, c, c.copy(), f)


def plain_box32(seed: int = 0) -> Problem:
    """Single 32^3 unit-spaced box, f ~ U[-1, 1], G_L and E(0.1), FP64."""
    p = uniform_box(32, (1, 1, 1), seed)
    p.name = "box32_fp64"
    p.alphas = (0.1,)
    return p


def blob_field(b: int, coords: np.ndarray, centres: np.ndarray, amps: np.ndarray, sigma: float) -> np.ndarray:
    """sum_j a_j exp(-|x - c_j|^2 / (2 sigma^2)) at the lattice points of the blocks."""
    pts = block_point_coords(b, coords).reshape(-1, 3).astype(np.float64)
    out = np.zeros(pts.shape[0])
    for c, a in zip(centres, amps):
        d2 = ((pts - c) ** 2).sum(axis=1)
        out += a * np.exp(-d2 / (2.0 * sigma * sigma))
    return out.reshape(coords.shape[0], b ** 3)


def dense_blobs(n: int = 128, b: int = 32, seed: int = 1, nblobs: int = 8, sigma: float = 6.0) -> Problem:
    """Dense n^3 box; f = sum of Gaussian blobs (sigma cells, N(0,1) amplitudes,
    centres uniform in the inner (n - 32)^3)."""
    rng = np.random.default_rng(seed)
    nb = n // b
    c = box_blocks(nb, nb, nb)
    margin = 16.0
    centres = rng.uniform(margin, n - margin, size=(nblobs, 3))
    amps = rng.normal(size=nblobs)
    f = blob_field(b, c, centres, amps, sigma)[None, None]
    return Problem(f"dense{n}_blobs", b, c, c.copy(), f, alphas=(0.05, 0.5, 2.0),
                   meta={"centres": centres, "amps": amps, "sigma": sigma})


def sphere_wake_blocks(b: int = 16, radius_blocks: float = 4.0, wake_len: float = 12.0,
                       wake_radius: float = 3.0) -> np.ndarray:
    """Blocks whose centre lies within ``radius_blocks`` of the origin, plus a
    wake cylinder x in [0, wake_len], radius ``wake_radius`` (block units)."""
    R = int(math.ceil(max(radius_blocks, wake_len))) + 1
    r = np.arange(-R, R + 1)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    cx, cy, cz = x + 0.5, y + 0.5, z + 0.5
    ball = cx ** 2 + cy ** 2 + cz ** 2 <= radius_blocks ** 2
    wake = (cx >= 0) & (cx <= wake_len) & (cy ** 2 + cz ** 2 <= wake_radius ** 2)
    m = ball | wake
    return np.stack([x[m], y[m], z[m]], axis=1).astype(np.int32)


def sphere_ib(seed: int = 2, b: int = 16, level: int = 5, radius_cells: float = 20.0) -> Problem:
    """Block-adaptive sphere: sphere + wake active set, 3-component sources
    spread from 20*4^(level-1) icosphere markers with N(0,1) forces."""
    rng = np.random.default_rng(seed)
    tgt = sphere_wake_blocks(b)
    X = icosphere_markers(level) * radius_cells
    F = rng.normal(size=X.shape)
    src = blocks_touched(b, X)
    tset = {tuple(c) for c in tgt.tolist()}
    src = np.array([c for c in src.tolist() if tuple(c) in tset], dtype=np.int32)
    f = spread_to_blocks(b, src, X, F)[None]
    return Problem("sphere_ib", b, src, tgt, f, alphas=(0.25,), meta={"markers": X.shape[0]})


def plate_problem(rng, nb_target: int, b: int, ar: int, chord: float = 40.0) -> Problem:
    """One flat-plate problem with about ``nb_target`` active blocks: the plate's
    own blocks plus a downstream wake grown to the drawn count."""
    spacing = 1.05
    X = None
    src = None
    c = chord
    for _ in range(20):
        X = plate_markers(c, ar * c, spacing, 30.0)
        src = blocks_touched(b, X)
        if src.shape[0] <= max(1, nb_target):
            break
        c *= 0.8
    # wake: blocks downstream (+x) of the plate's block bounding box, nearest first
    lo = src.min(axis=0)
    hi = src.max(axis=0)
    need = max(0, nb_target - src.shape[0])
    sset = {tuple(v) for v in src.tolist()}
    cand = []
    span = hi - lo + 1
    L = int(math.ceil(need / max(1, span[1] * span[2]))) + 2
    for xx in range(lo[0], hi[0] + 1 + L):
        for yy in range(lo[1] - 1, hi[1] + 2):
            for zz in range(lo[2], hi[2] + 1):
                if (xx, yy, zz) not in sset:
                    cand.append((xx, yy, zz))
    cand = np.array(cand, dtype=np.int64).reshape(-1, 3)
    if cand.shape[0]:
        ctr = (lo + hi) / 2.0
        d = np.abs(cand[:, 0] - ctr[0]) + 2.0 * np.abs(cand[:, 1] - ctr[1]) + 0.5 * np.abs(cand[:, 2] - ctr[2])
        cand = cand[np.argsort(d, kind="stable")][:need]
    tgt = np.concatenate([src, cand.astype(np.int32)]) if cand.shape[0] else src.copy()
    F = rng.normal(size=X.shape)
    f = spread_to_blocks(b, src, X, F)[None]
    return Problem(f"plate_ar{ar}", b, src.astype(np.int32), tgt.astype(np.int32), f, alphas=(0.25,),
                   meta={"chord": c, "markers": X.shape[0]})


def plate_batch(seed: int = 3, nprob: int = 64, b: int = 16, nb_lo: int = 8, nb_hi: int = 1200) -> list:
    """Independent flat-plate problems, active block counts log-uniform in
    [nb_lo, nb_hi], AR in {1, 2, 4} round robin, G_L then E(0.25)."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(nb_lo), math.log(nb_hi), size=nprob)).astype(int)
    probs = []
    for i, n in enumerate(counts):
        probs.append(plate_problem(rng, int(n), b, (1, 2, 4)[i % 3]))
    return probs


def wake_mask_blocks(nbx: int = 16, nby: int = 8, nbz: int = 8, frac: float = 0.4) -> np.ndarray:
    """Sphere-plus-wake mask on an nbx x nby x nbz block grid keeping about
    ``frac`` of the blocks: a ball around (nbx/4, nby/2, nbz/2) joined to a
    downstream cylinder whose radius is grown until the fraction is reached."""
    z, y, x = np.meshgrid(np.arange(nbz), np.arange(nby), np.arange(nbx), indexing="ij")
    cx, cy, cz = x + 0.5, y + 0.5, z + 0.5
    sx, sy, sz = nbx / 4.0, nby / 2.0, nbz / 2.0
    target = frac * nbx * nby * nbz
    best = None
    for rad in np.linspace(0.5, max(nby, nbz), 200):
        ball = (cx - sx) ** 2 + (cy - sy) ** 2 + (cz - sz) ** 2 <= (1.2 * rad) ** 2
        wake = (cx >= sx) & ((cy - sy) ** 2 + (cz - sz) ** 2 <= rad ** 2)
        m = ball | wake
        if best is None or abs(m.sum() - target) < abs(best.sum() - target):
            best = m
    return np.stack([x[best], y[best], z[best]], axis=1).astype(np.int32)


def curl_blob_field(b: int, coords: np.ndarray, centres: np.ndarray, amps: np.ndarray, sigma: float) -> np.ndarray:
    """Face-lattice samples of curl(A), A = sum_j a_j exp(-|x - c_j|^2/(2 sigma^2))
    (vector amplitudes a_j): returns [3][nblk][b^3].  Each Gaussian factorises
    over the three axes, so it is evaluated as per-axis factors broadcast over
    the blocks."""
    coords = np.asarray(coords, dtype=np.int64)
    nb = coords.shape[0]
    r = np.arange(b, dtype=np.float64)
    out = np.zeros((3, nb, b, b, b))
    s2 = sigma * sigma
    for k in range(3):
        off = face_offset(k)
        # axis positions of every block: [nblk][b]
        pos = [coords[:, ax:ax + 1] * b + r[None, :] + off[ax] for ax in range(3)]
        i, j = (k + 1) % 3, (k + 2) % 3
        for c, a in zip(centres, amps):
            # blocks farther than 10 sigma on some axis get less than e^-50: skip them
            near = np.ones(nb, dtype=bool)
            for ax in range(3):
                near &= np.abs(pos[ax] - c[ax]).min(axis=1) < 10.0 * sigma
            if not near.any():
                continue
            d = [pos[ax][near] - c[ax] for ax in range(3)]
            g = [np.exp(-d[ax] ** 2 / (2.0 * s2)) for ax in range(3)]
            # (curl A)_k = d_i A_j - d_j A_i,  d_i exp(...) = -(x_i - c_i)/sigma^2 exp(...)
            term_i = [g[0], g[1], g[2]]
            term_i[i] = -d[i] * g[i] / s2          # d_i of the Gaussian
            term_j = [g[0], g[1], g[2]]
            term_j[j] = -d[j] * g[j] / s2          # d_j of the Gaussian
            ti = term_i[2][:, :, None, None] * term_i[1][:, None, :, None] * term_i[0][:, None, None, :]
            tj = term_j[2][:, :, None, None] * term_j[1][:, None, :, None] * term_j[0][:, None, None, :]
            out[k][near] += a[j] * ti - a[i] * tj
    return out.reshape(3, nb, b ** 3)


def wake_domain(seed: int = 4, b: int = 32, nrhs: int = 4, shape=(512, 256, 256), nblobs: int = 32,
                sigma: float = 10.0) -> Problem:
    """Large wake domain: sphere-plus-wake mask (~40% of the blocks) of a
    shape[0] x shape[1] x shape[2] lattice, 3-component smooth vortical sources
    (curl of a Gaussian-blob vector potential), ``nrhs`` right-hand sides."""
    nb = [s // b for s in shape]
    c = wake_mask_blocks(*nb)
    rng = np.random.default_rng(seed)
    lo = c.min(axis=0) * b
    hi = (c.max(axis=0) + 1) * b
    f = np.empty((nrhs, 3, c.shape[0], b ** 3))
    for r in range(nrhs):
        centres = rng.uniform(lo, hi, size=(nblobs, 3))
        amps = rng.normal(size=(nblobs, 3))
        f[r] = curl_blob_field(b, c, centres, amps, sigma)
    return Problem("wake_domain", b, c, c.copy(), f, meta={"shape": shape})


def random_sparse(seed: int, b: int = 16, nsrc: int = 5, ntgt: int = 7, extent=(4, 3, 3),
                  nrhs: int = 1, ncomp: int = 1) -> Problem:
    """Small random block sets (possibly disjoint src/tgt) with U[-1,1] sources,
    for element-by-element parity at oracle-friendly sizes."""
    rng = np.random.default_rng(seed)
    src = random_blockset(rng, nsrc, extent)
    tgt = random_blockset(rng, ntgt, extent, origin=(rng.integers(-1, 2), rng.integers(-1, 2), 0))
    f = rng.uniform(-1.0, 1.0, size=(nrhs, ncomp, nsrc, b ** 3))
    return Problem("random_sparse", b, src, tgt, f)
