"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds no BDDC-SO arithmetic.  It only draws the problem data the
paper's experiments are defined on (Section 5): the unit-cube hexahedral mesh
size, the per-axis subdomain cut planes, the subobject size L, the per-element
diffusion coefficient alpha (Remark 1) and the right-hand side vector b of the
Q1 load functional <F, v> (Section 2, eq. weakform).

Random numbers come from one counter-based generator, splitmix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
draw k of stream `seed` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15) and the
double in [0, 1) is its top 53 bits times 2^-53.  Normals use Box-Muller on
consecutive pairs.

Layouts (shared with the C ABI):
  * alpha: float64, nx*ny*nz, element (i, j, k) at i + nx*(j + ny*k).
  * node vectors: float64, (nx+1)*(ny+1)*(nz+1), node (i, j, k) at
    i + (nx+1)*(j + (ny+1)*k); entries on the Dirichlet boundary are 0.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 2001072890
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the splitmix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64 draws."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]            # (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# --------------------------------------------------------------------------
# cut planes
# --------------------------------------------------------------------------

def uniform_cuts(n: int, parts: int) -> List[int]:
    """Interior cut planes (element indices) splitting n elements into equal parts."""
    if n % parts:
        raise ValueError("n must be divisible by parts")
    w = n // parts
    return [w * i for i in range(1, parts)]


def jittered_cuts(n: int, parts: int, seed: int, jitter: int = 3) -> List[int]:
    """Cuts c_i = (n/parts)*i + d_i with d_0 = 0 and d_i drawn uniformly from the
    integers v in [-jitter, jitter] with |v - d_{i-1}| <= jitter, so that every
    subdomain width lies in [n/parts - 2*jitter, n/parts + 2*jitter]."""
    w = n // parts
    u = uniform01(seed, parts - 1)
    d_prev = 0
    cuts = []
    for i in range(1, parts):
        lo = max(-jitter, d_prev - jitter)
        hi = min(jitter, d_prev + jitter)
        d = lo + min(int(u[i - 1] * (hi - lo + 1)), hi - lo)
        cuts.append(w * i + d)
        d_prev = d
    # the last subdomain width is w - d_{parts-1}, within the same bounds
    return cuts


# --------------------------------------------------------------------------
# coefficients
# --------------------------------------------------------------------------

def alpha_constant(nx: int, ny: int, nz: int, value: float = 1.0) -> np.ndarray:
    return np.full(nx * ny * nz, value, dtype=np.float64)


def alpha_blocks(nx: int, ny: int, nz: int, block: int, high: float, p: float,
                 seed: int) -> np.ndarray:
    """alpha constant on block^3 element blocks: `high` where a uniform draw of
    the block is below p, else 1 (blocks numbered x fastest)."""
    bx, by, bz = nx // block, ny // block, nz // block
    u = uniform01(seed, bx * by * bz).reshape(bz, by, bx)
    blk = np.where(u < p, high, 1.0)
    a = np.repeat(np.repeat(np.repeat(blk, block, axis=0), block, axis=1), block, axis=2)
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def alpha_loguniform(nx: int, ny: int, nz: int, lo_exp: float, hi_exp: float,
                     seed: int) -> np.ndarray:
    """alpha_e = 10^U[lo_exp, hi_exp] per element."""
    u = uniform01(seed, nx * ny * nz)
    return 10.0 ** (lo_exp + (hi_exp - lo_exp) * u)


def gaussian_field(nx: int, ny: int, nz: int, corr_len: float, seed: int,
                   h: Optional[float] = None) -> np.ndarray:
    """Zero-mean unit-variance Gaussian field at element centroids with the
    separable squared-exponential covariance exp(-|x-y|^2 / (2 l^2)), sampled as
    (V_z S_z^1/2 (x) V_y S_y^1/2 (x) V_x S_x^1/2) xi with xi ~ N(0, I) and
    V S V^T the eigendecomposition of each 1-D covariance (negative eigenvalues
    of the numerically indefinite matrix clipped to 0)."""
    h = h if h is not None else 1.0 / nx
    factors = []
    for n in (nx, ny, nz):
        x = (np.arange(n) + 0.5) * h
        c = np.exp(-((x[:, None] - x[None, :]) ** 2) / (2.0 * corr_len ** 2))
        s, v = np.linalg.eigh(c)
        factors.append(v * np.sqrt(np.clip(s, 0.0, None))[None, :])
    xi = normals(seed, nx * ny * nz).reshape(nz, ny, nx)
    fx, fy, fz = factors
    g = np.einsum("ia,abc->ibc", fz, xi)
    g = np.einsum("jb,ibc->ijc", fy, g)
    g = np.einsum("kc,ijc->ijk", fx, g)
    return np.ascontiguousarray(g).reshape(-1)


# --------------------------------------------------------------------------
# right-hand side: b_n = integral of f * phi_n over the mesh (Q1 hat functions)
# --------------------------------------------------------------------------

def _interior_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    m[1:nz, 1:ny, 1:nx] = True
    return m


def rhs_constant(nx: int, ny: int, nz: int, h: float, f: float = 1.0) -> np.ndarray:
    """b for constant f: every interior hat function integrates to h^3 exactly."""
    b = np.where(_interior_mask(nx, ny, nz), f * h ** 3, 0.0)
    return b.reshape(-1)


def rhs_quadrature(nx: int, ny: int, nz: int, h: float, f) -> np.ndarray:
    """b_n = sum over elements of the 2x2x2 Gauss-Legendre rule applied to
    f * phi_n (f vectorised over x, y, z arrays)."""
    g = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    phi = np.stack([1.0 - g, g])           # phi[a, q]: 1-D hat a at Gauss point q
    b = np.zeros((nz + 1, ny + 1, nx + 1))
    ex = np.arange(nx)[None, None, :]
    ey = np.arange(ny)[None, :, None]
    ez = np.arange(nz)[:, None, None]
    for qz in range(2):
        for qy in range(2):
            for qx in range(2):
                fv = f((ex + g[qx]) * h, (ey + g[qy]) * h, (ez + g[qz]) * h) * (h ** 3 / 8.0)
                for az in range(2):
                    for ay in range(2):
                        for ax in range(2):
                            w = phi[ax, qx] * phi[ay, qy] * phi[az, qz]
                            b[az:az + nz, ay:ay + ny, ax:ax + nx] += w * fv
    b[~_interior_mask(nx, ny, nz)] = 0.0
    return b.reshape(-1)


def manufactured_u(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def manufactured_f(x, y, z):
    """f = -lap(u) for u = sin(pi x) sin(pi y) sin(pi z) with alpha = 1."""
    return 3.0 * np.pi ** 2 * manufactured_u(x, y, z)


def random_node_vector(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """Uniform(-1, 1) on interior nodes, 0 on the Dirichlet boundary."""
    v = 2.0 * uniform01(seed, (nx + 1) * (ny + 1) * (nz + 1)) - 1.0
    v = v.reshape(nz + 1, ny + 1, nx + 1)
    v[~_interior_mask(nx, ny, nz)] = 0.0
    return v.reshape(-1)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    cuts: List[List[int]]        # interior cut planes per axis (x, y, z)
    L: int                       # subobject size in elements
    alpha: np.ndarray            # per element, x fastest
    b: np.ndarray                # per node, x fastest, 0 on the boundary
    weights: str = "card"        # "card" (eq. W) or "rho" (Remark 1)
    rtol: float = 1e-10
    precision: str = "fp64"      # "fp64" or "mixed"
    selection: str = "vef"
    piece: Optional[np.ndarray] = None   # per-element sub-subdomain labels (None: boxes of size L)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_free(self) -> int:
        return (self.nx - 1) * (self.ny - 1) * (self.nz - 1)

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * self.nz


def channel_mask(nx: int, ny: int, nz: int, per_axis: int, width: int, seed: int,
                 cuts: Optional[Sequence[Sequence[int]]] = None) -> np.ndarray:
    """Per-element indicator (x fastest) of a system of straight channels:
    per_axis bars of width x width elements running through the whole mesh
    along each axis, at seeded transverse positions (the channels geometry of
    Section 5.2 is only in a missing figure; this one is synthetic).  With
    cuts, every bar lies inside one slab of each transverse axis, at least one
    element away from its cut planes: a bar that straddled a cut plane
    parallel to it would meet its continuation in a diagonal subdomain only
    along an edge, leaving that pair of channel pieces without an acceptable
    path under face constraints (remark after Theorem 1)."""
    n = (nx, ny, nz)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    u = uniform01(seed, 6 * per_axis)

    def position(t, v):
        if cuts is None:
            return 1 + int(v * (n[t] - width - 1))
        b = [0] + list(cuts[t]) + [n[t]]
        room = [(lo + 1, hi - 1 - width) for lo, hi in zip(b[:-1], b[1:]) if hi - 1 - width >= lo + 1]
        if not room:
            raise ValueError("slabs too thin for channels of this width")
        k = min(int(v * len(room)), len(room) - 1)
        lo, hi = room[k]
        w = v * len(room) - k
        return lo + min(int(w * (hi - lo + 1)), hi - lo)

    q = 0
    for d in range(3):
        t1, t2 = (d + 1) % 3, (d + 2) % 3
        for _ in range(per_axis):
            a, b = position(t1, u[q]), position(t2, u[q + 1])
            q += 2
            sl = [slice(None)] * 3            # array axes are (z, y, x)
            sl[2 - t1] = slice(a, a + width)
            sl[2 - t2] = slice(b, b + width)
            mask[tuple(sl)] = True
    return mask.reshape(-1)


def material_pieces(nx: int, ny: int, nz: int, cuts: Sequence[Sequence[int]], mask: np.ndarray) -> np.ndarray:
    """Per-element sub-subdomain labels splitting every subdomain of the box
    partition into its background and its channel part (Section 5.2: two
    sub-subdomains per subdomain), numbered densely in the order of
    2 subdomain + indicator."""
    def slab(n, c):
        return np.searchsorted(np.asarray(c, dtype=np.int64), np.arange(n), side="right")
    sx, sy, sz = slab(nx, cuts[0]), slab(ny, cuts[1]), slab(nz, cuts[2])
    nsx, nsy = len(cuts[0]) + 1, len(cuts[1]) + 1
    sub = sx[None, None, :] + nsx * (sy[None, :, None] + nsy * sz[:, None, None])
    key = 2 * sub.reshape(-1) + np.asarray(mask, dtype=np.int64).reshape(-1)
    return np.unique(key, return_inverse=True)[1].reshape(-1).astype(np.int64)


def channels_problem(n: int = 40, parts: int = 4, ell: float = 4.0, per_axis: int = 3, width: int = 2,
                     seed: int = 0, sub_partition: str = "material", selection: str = "f", **kw) -> Problem:
    """The channels experiment of Section 5.2 on synthetic channels: n^3
    hexahedra, parts^3 box subdomains, alpha = 10^ell in the channels and 1
    elsewhere, f = 1, rho-weights (Remark 1), PCG to rtol 1e-6.
    sub_partition "material": Theta-hat = {background, channels} per
    subdomain (BDDC-SO); "none": Theta-hat = Theta (standard BDDC)."""
    cuts = [uniform_cuts(n, parts)] * 3
    mask = channel_mask(n, n, n, per_axis, width, BASE_SEED + 100 + seed, cuts)
    alpha = np.where(mask, 10.0 ** ell, 1.0)
    if sub_partition == "material":
        piece, L = material_pieces(n, n, n, cuts, mask), n
    elif sub_partition == "none":
        piece, L = None, n
    else:
        raise ValueError(sub_partition)
    kw.setdefault("rtol", 1e-6)
    kw.setdefault("weights", "rho")
    return box_problem(n, n, n, cuts, L, alpha=alpha, name=f"channels{n}_l{ell:g}", selection=selection,
                       piece=piece, **kw)


def box_problem(nx: int, ny: int, nz: int, cuts: Sequence[Sequence[int]], L: int,
                alpha: Optional[np.ndarray] = None, rhs: str = "one",
                name: str = "box", **kw) -> Problem:
    """A Poisson-type problem on [0, nx h] x [0, ny h] x [0, nz h] with h = 1/nx."""
    h = 1.0 / nx
    if alpha is None:
        alpha = alpha_constant(nx, ny, nz)
    if rhs == "one":
        b = rhs_constant(nx, ny, nz, h)
    elif rhs == "manufactured":
        b = rhs_quadrature(nx, ny, nz, h, manufactured_f)
    else:
        raise ValueError(rhs)
    return Problem(name, nx, ny, nz, h, [list(c) for c in cuts], L, alpha, b, **kw)


def workload(index: int, L: Optional[int] = None, precision: Optional[str] = None) -> Problem:
    """The five synthetic workloads (0-based index):

    0: 16^3, 2^3 subdomains of 8^3, L=4, alpha=1, f=1, FP64, rtol 1e-10.
    1: 48^3, 4^3 subdomains of 12^3, L in {4, 2}, alpha=1, manufactured f,
       FP64 or mixed, rtol 1e-10.
    2: 96^3, 8^3 subdomains of 12^3, L=4, alpha in {1, 1e6} per 4^3 block
       (p=0.3), rho-weights, f=1, mixed, rtol 1e-8.
    3: 128^3, 16^3 jittered subdomains (widths 5..11), L in {2, 4},
       alpha = 10^U[-2,2] per element, f=1, mixed, rtol 1e-10.
    4: 64^3, 4^3 subdomains of 16^3, L=4, log alpha Gaussian field
       (correlation length 0.1), f=1, FP64 (adjoint workload).
    """
    seed = BASE_SEED + index + 1
    if index == 0:
        n = 16
        return box_problem(n, n, n, [uniform_cuts(n, 2)] * 3, L or 4, name="poisson16",
                           rtol=1e-10, precision=precision or "fp64")
    if index == 1:
        n = 48
        return box_problem(n, n, n, [uniform_cuts(n, 4)] * 3, L or 4, rhs="manufactured",
                           name="poisson48", rtol=1e-10, precision=precision or "mixed")
    if index == 2:
        n = 96
        a = alpha_blocks(n, n, n, 4, 1e6, 0.3, seed)
        return box_problem(n, n, n, [uniform_cuts(n, 8)] * 3, L or 4, alpha=a,
                           name="channels96", weights="rho", rtol=1e-8,
                           precision=precision or "mixed")
    if index == 3:
        n = 128
        cuts = [jittered_cuts(n, 16, seed + d) for d in range(3)]
        a = alpha_loguniform(n, n, n, -2.0, 2.0, seed + 3)
        return box_problem(n, n, n, cuts, L or 4, alpha=a, name="jitter128",
                           rtol=1e-10, precision=precision or "mixed")
    if index == 4:
        n = 64
        a = np.exp(gaussian_field(n, n, n, 0.1, seed))
        return box_problem(n, n, n, [uniform_cuts(n, 4)] * 3, L or 4, alpha=a,
                           name="adjoint64", rtol=1e-10, precision=precision or "fp64")
    raise ValueError(index)


def observation_field_alpha(n: int = 64, index: int = 4) -> np.ndarray:
    """The second coefficient field alpha' whose forward solution, perturbed by
    1% noise (observation_noise), is the observation u_obs of the adjoint workload."""
    return np.exp(gaussian_field(n, n, n, 0.1, BASE_SEED + index + 1 + 1))


def observation_noise(n_nodes: int, index: int = 4) -> np.ndarray:
    return normals(BASE_SEED + index + 1 + 2, n_nodes)


def fd_directions(n_elems: int, count: int = 20, index: int = 4) -> np.ndarray:
    """count seeded N(0,1) directions in theta = log(alpha), one row each."""
    return normals(BASE_SEED + index + 1 + 3, count * n_elems).reshape(count, n_elems)
