"""Seeded synthetic inputs for the Wilson-clover quark solver.

This module generates the gauge fields, sources and batch draws that stand in
for the paper's workload (a random gauge configuration on a 32^4 lattice and a
Gaussian noise source, Sec. 5).  The authors' configuration is not available,
so every input is drawn here from a seed.

It is shared by the CPU oracle's tests, the GPU tests and the benchmark, and it
holds none of the method's arithmetic: no Dirac operator, clover term, Schwarz
step or Krylov solver lives here.  It only produces arrays.

Random numbers
--------------
The generator is SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Its n-th output (n = 0, 1, ...)
for seed ``s`` is the 64-bit finaliser applied to ``s + (n + 1) * 0x9E3779B97F4A7C15``,
so any output can be computed directly from its index; this makes the stream
vectorisable in numpy and identical on every machine.

* uniform u_n = ((out_n >> 11) + 0.5) * 2^-53, in the open interval (0, 1);
* normals come in Box-Muller pairs: for pair j, u1 = u_{2j}, u2 = u_{2j+1},
  z_{2j} = sqrt(-2 ln u1) cos(2 pi u2), z_{2j+1} = sqrt(-2 ln u1) sin(2 pi u2).

Layouts (canonical, FP64 complex)
---------------------------------
* site index  i = x + Lx (y + Ly (z + Lz t)), dims given as (Lx, Ly, Lz, Lt);
* spinor      complex128 [V][spin 4][colour 3];
* gauge field complex128 [V][mu 4 = x,y,z,t][row 3][col 3].

Gauge links: for each site in lexicographic order and each mu, 18 normals fill
a 3x3 complex matrix M row-major (real part then imaginary part of each
entry); H = (M + M^dag)/2 - tr(.)/3, a traceless Hermitian matrix; the link is
U = exp(i eps H), computed from the Hermitian eigendecomposition of H.  Then U
is unitary and det U = 1 to rounding.

Sources: per site, spin and colour, the real and then the imaginary part are
independent N(0, 1) draws.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniforms",
    "normals",
    "volume",
    "gauge_field",
    "unit_gauge",
    "random_su3",
    "gaussian_source",
    "point_source",
    "uneven_batch",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """n-th SplitMix64 outputs for ``seed`` at the given uint64 indices."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in (0, 1) for stream indices start .. start+count-1."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    bits = splitmix64(seed, idx) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(seed: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` N(0,1) draws of the stream for ``seed``, beginning at normal
    number ``start`` (which must be even, so that Box-Muller pairs stay whole)."""
    if start % 2:
        raise ValueError("start must be even")
    out = np.empty(count, dtype=np.float64)
    npairs = (count + 1) // 2
    p0 = start // 2
    done = 0
    for c0 in range(0, npairs, _CHUNK):
        c1 = min(npairs, c0 + _CHUNK)
        u = uniforms(seed, 2 * (p0 + c0), 2 * (c1 - c0)).reshape(-1, 2)
        r = np.sqrt(-2.0 * np.log(u[:, 0]))
        ang = 2.0 * np.pi * u[:, 1]
        z = np.empty((c1 - c0, 2), dtype=np.float64)
        z[:, 0] = r * np.cos(ang)
        z[:, 1] = r * np.sin(ang)
        z = z.reshape(-1)
        take = min(z.size, count - done)
        out[done:done + take] = z[:take]
        done += take
    return out


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def _exp_i_eps_h(m: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps H) with H the traceless Hermitian part of each 3x3 matrix m."""
    h = 0.5 * (m + np.conj(np.swapaxes(m, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return (v * ph[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) gauge field U = exp(i eps H), complex128 [V][4][3][3]."""
    vol = volume(dims)
    nmat = vol * 4
    u = np.empty((nmat, 3, 3), dtype=np.complex128)
    step = 1 << 19
    for m0 in range(0, nmat, step):
        m1 = min(nmat, m0 + step)
        z = normals(seed, (m1 - m0) * 18, start=m0 * 18).reshape(m1 - m0, 3, 3, 2)
        m = z[..., 0] + 1j * z[..., 1]
        u[m0:m1] = _exp_i_eps_h(m, eps)
    return u.reshape(vol, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    """Free field: every link the identity."""
    vol = volume(dims)
    u = np.zeros((vol, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def random_su3(count: int, seed: int, eps: float = 1.0) -> np.ndarray:
    """``count`` random SU(3) matrices exp(i eps H) (used as gauge transforms)."""
    z = normals(seed, count * 18).reshape(count, 3, 3, 2)
    return _exp_i_eps_h(z[..., 0] + 1j * z[..., 1], eps)


def gaussian_source(dims, seed: int) -> np.ndarray:
    """Complex Gaussian spinor, complex128 [V][4][3]."""
    vol = volume(dims)
    z = normals(seed, vol * 24).reshape(vol, 4, 3, 2)
    return z[..., 0] + 1j * z[..., 1]


def point_source(dims, spin: int, colour: int, site: int = 0) -> np.ndarray:
    """Unit point source delta(x, site) delta(s, spin) delta(c, colour)."""
    vol = volume(dims)
    s = np.zeros((vol, 4, 3), dtype=np.complex128)
    s[site, spin, colour] = 1.0
    return s


UNEVEN_SHAPES = ((8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (8, 8, 8, 24), (24, 24, 24, 24))


def uneven_batch(n: int, master_seed: int = 1):
    """Draw ``n`` independent systems for an uneven batch.

    Each system gets a lattice shape from UNEVEN_SHAPES, eps ~ U[0.2, 0.35],
    kappa ~ U[0.11, 0.124] and its own gauge and source seeds, all drawn from
    the stream of ``master_seed`` (four uniforms per system).
    """
    u = uniforms(master_seed, 0, 4 * n).reshape(n, 4)
    out = []
    for k in range(n):
        shape = UNEVEN_SHAPES[min(int(u[k, 0] * len(UNEVEN_SHAPES)), len(UNEVEN_SHAPES) - 1)]
        out.append({
            "dims": shape,
            "eps": 0.2 + 0.15 * float(u[k, 1]),
            "kappa": 0.11 + 0.014 * float(u[k, 2]),
            "c_sw": 1.0,
            "gauge_seed": 1000 + 2 * k,
            "source_seed": 1001 + 2 * k,
        })
    return out
