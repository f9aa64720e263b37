"""Seeded synthetic inputs shaped like the random sparse tensors of the paper's experiments.

This module is shared by the CPU oracle's tests, the GPU parity tests and the benchmark. It
holds no arithmetic of the decomposition methods: it only draws random numbers and lays them
out as COO tensors and raw uniform matrices.

Random source: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: output i of a stream with seed s
is mix(s + (i+1) * 0x9E3779B97F4A7C15).  Doubles take the top 53 bits: (u >> 11) * 2**-53.

Tensor model (Section "Varying Tensor Sizes" and the appendix generator: random sparse third
order tensors with values uniform on [0, 1]).  The paper draws a Bernoulli cell mask; here the
number of nonzeros is exact: candidate linear indices floor(u * N / 2**64) are drawn in stream
order and the first `nnz` distinct ones are kept, in acceptance order (so COO order is random
and the sort in the CSF build is exercised).  Value i is uniform01 of draw i of a second stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 5678  # the seed of the paper's appendix test driver


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 stream with the given seed (uint64)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * GOLDEN)


def splitmix64_scalar(seed: int) -> int:
    """First output of the stream with the given seed; used to derive sub-seeds."""
    return int(splitmix64(seed, 1)[0])


def uniform01(u: np.ndarray) -> np.ndarray:
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _mulhi(u: np.ndarray, n: int) -> np.ndarray:
    """floor(u * n / 2**64) for uint64 u and 0 < n < 2**63, via 32-bit limbs (exact)."""
    mask = np.uint64(0xFFFFFFFF)
    n = np.uint64(n)
    n_lo, n_hi = n & mask, n >> np.uint64(32)
    u_lo, u_hi = u & mask, u >> np.uint64(32)
    with np.errstate(over="ignore"):
        lolo = u_lo * n_lo
        hilo = u_hi * n_lo
        lohi = u_lo * n_hi
        hihi = u_hi * n_hi
        mid = (lolo >> np.uint64(32)) + (hilo & mask) + (lohi & mask)
        return hihi + (hilo >> np.uint64(32)) + (lohi >> np.uint64(32)) + (mid >> np.uint64(32))


@dataclass
class CooTensor:
    dims: tuple          # (I1, I2, I3)
    idx: np.ndarray      # int32 [3, nnz], 0-based
    val: np.ndarray      # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])


def config_seed(config_id: int, base: int = BASE_SEED) -> int:
    return splitmix64_scalar(base ^ config_id)


def random_sparse_tensor(dims, nnz: int, seed: int) -> CooTensor:
    """Exactly `nnz` distinct uniformly random coordinates, values U[0,1) (see module doc)."""
    dims = tuple(int(d) for d in dims)
    N = dims[0] * dims[1] * dims[2]
    if nnz > N:
        raise ValueError("nnz exceeds the number of cells")
    s_coord = splitmix64_scalar(seed ^ 0x636F6F7264)   # "coord"
    s_val = splitmix64_scalar(seed ^ 0x76616C)         # "val"
    chosen = np.empty(0, dtype=np.int64)
    drawn = 0
    while chosen.shape[0] < nnz:
        need = nnz - chosen.shape[0]
        batch = max(1024, int(need * (1.0 + 2.0 * nnz / N)) + 64)
        lin = _mulhi(splitmix64(s_coord, batch, offset=drawn), N).astype(np.int64)
        drawn += batch
        allc = np.concatenate([chosen, lin])
        _, first = np.unique(allc, return_index=True)
        first.sort()                       # acceptance order = first occurrence in stream order
        chosen = allc[first][:nnz]
    I2I3 = dims[1] * dims[2]
    i = chosen // I2I3
    j = (chosen // dims[2]) % dims[1]
    k = chosen % dims[2]
    idx = np.stack([i, j, k]).astype(np.int32)
    val = uniform01(splitmix64(s_val, nnz))
    return CooTensor(dims, idx, val)


def uniform_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """rows x cols matrix of U[0,1) draws filled row-major (the raw draw behind SP's random C)."""
    return uniform01(splitmix64(seed, rows * cols)).reshape(rows, cols)


def paper_config(name: str):
    """(dims, nnz, core) of the synthetic workloads, named by their sizes."""
    table = {
        "100^3/1e5/J10": ((100, 100, 100), 100_000, (10, 10, 10)),
        "1000^3/1e7/J50": ((1000, 1000, 1000), 10_000_000, (50, 50, 50)),
        "2000^3/4e7/J100": ((2000, 2000, 2000), 40_000_000, (100, 100, 100)),
        "500^3/2.5e6/J50": ((500, 500, 500), 2_500_000, (50, 50, 50)),
        "500^3/2.5e6/J25-50-100": ((500, 500, 500), 2_500_000, (25, 50, 100)),
        "500^3/2.5e6/J10-50-250": ((500, 500, 500), 2_500_000, (10, 50, 250)),
        "500^3/2.5e6/J250-50-10": ((500, 500, 500), 2_500_000, (250, 50, 10)),
        "250^3/10%/J25": ((250, 250, 250), 1_562_500, (25, 25, 25)),
        "100x110x120/10%/J10-11-12": ((100, 110, 120), 132_000, (10, 11, 12)),
    }
    return table[name]


def batched_configs(count: int, seed: int):
    """Per-tensor (dims, nnz, core) of the batched workload: each dim uniform integer in
    [30, 300], density log-uniform in [1%, 20%], each core dim uniform integer in [4, 32]
    and at most its tensor dim."""
    u = uniform01(splitmix64(seed, count * 7)).reshape(count, 7)
    out = []
    for t in range(count):
        dims = tuple(30 + int(u[t, a] * 271) for a in range(3))
        dens = math.exp(math.log(0.01) + u[t, 3] * (math.log(0.20) - math.log(0.01)))
        N = dims[0] * dims[1] * dims[2]
        nnz = max(1, int(round(dens * N)))
        core = tuple(min(dims[a], 4 + int(u[t, 4 + a] * 29)) for a in range(3))
        out.append((dims, nnz, core))
    return out


def planted_tensor(dims, core, support, seed: int):
    """Sparse tensor of exact multilinear rank `core`: X = G x1 A x2 B x3 C with random G and
    orthonormal factors whose rows vanish outside random support sets of the given sizes.
    Returns (CooTensor, G, [A, B, C]).  Orthonormalisation uses numpy's QR of a random
    Gaussian block; this is input construction, not a step of any decomposition method."""
    rng_u = uniform01(splitmix64(seed, 1 << 20))
    pos = [0]

    def take(n):
        a = rng_u[pos[0]:pos[0] + n]
        pos[0] += n
        return a

    def gauss(shape):
        n = int(np.prod(shape))
        u1, u2 = take(n), take(n)
        return (np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)

    factors, supports = [], []
    for a in range(3):
        sup = np.sort(np.argsort(take(dims[a]), kind="stable")[:support[a]])
        Q, _ = np.linalg.qr(gauss((support[a], core[a])))
        U = np.zeros((dims[a], core[a]))
        U[sup] = Q
        factors.append(U)
        supports.append(sup)
    G = gauss(tuple(core))
    sub = np.einsum("pqr,ip,jq,kr->ijk", G, factors[0][supports[0]],
                    factors[1][supports[1]], factors[2][supports[2]])
    ii, jj, kk = np.meshgrid(supports[0], supports[1], supports[2], indexing="ij")
    order = np.argsort(take(sub.size), kind="stable")   # scramble COO order
    idx = np.stack([ii.ravel(), jj.ravel(), kk.ravel()])[:, order].astype(np.int32)
    val = sub.ravel()[order].astype(np.float64)
    return CooTensor(tuple(dims), idx, val), G, factors


def random_sparse_tensor_n(dims, nnz: int, seed: int) -> CooTensor:
    """Order-N form of random_sparse_tensor (same scheme: the first `nnz` distinct linear
    indices floor(u * prod(dims) / 2**64) in stream order, values U[0,1) from a second stream;
    for N = 3 the result equals random_sparse_tensor's).  idx is int32 [N, nnz]."""
    dims = tuple(int(d) for d in dims)
    N = int(np.prod(dims))
    if nnz > N:
        raise ValueError("nnz exceeds the number of cells")
    s_coord = splitmix64_scalar(seed ^ 0x636F6F7264)
    s_val = splitmix64_scalar(seed ^ 0x76616C)
    chosen = np.empty(0, dtype=np.int64)
    drawn = 0
    while chosen.shape[0] < nnz:
        need = nnz - chosen.shape[0]
        batch = max(1024, int(need * (1.0 + 2.0 * nnz / N)) + 64)
        lin = _mulhi(splitmix64(s_coord, batch, offset=drawn), N).astype(np.int64)
        drawn += batch
        allc = np.concatenate([chosen, lin])
        _, first = np.unique(allc, return_index=True)
        first.sort()
        chosen = allc[first][:nnz]
    idx = np.empty((len(dims), nnz), dtype=np.int64)
    rem = chosen
    for a in reversed(range(len(dims))):
        idx[a] = rem % dims[a]
        rem = rem // dims[a]
    val = uniform01(splitmix64(s_val, nnz))
    return CooTensor(dims, idx.astype(np.int32), val)


def planted_tensor_n(dims, core, support, seed: int):
    """Order-N form of planted_tensor: X = G x1 U1 x2 U2 ... with random G and orthonormal
    factors whose rows vanish outside random support sets.  Returns (CooTensor, G, factors)."""
    rng_u = uniform01(splitmix64(seed, 1 << 21))
    pos = [0]

    def take(n):
        a = rng_u[pos[0]:pos[0] + n]
        pos[0] += n
        return a

    def gauss(shape):
        n = int(np.prod(shape))
        u1, u2 = take(n), take(n)
        return (np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)

    N = len(dims)
    factors, supports = [], []
    for a in range(N):
        sup = np.sort(np.argsort(take(dims[a]), kind="stable")[:support[a]])
        Q, _ = np.linalg.qr(gauss((support[a], core[a])))
        U = np.zeros((dims[a], core[a]))
        U[sup] = Q
        factors.append(U)
        supports.append(sup)
    G = gauss(tuple(core))
    sub = G
    for a in range(N):   # sub = G x_a U_a[support], mode by mode
        sub = np.moveaxis(np.tensordot(factors[a][supports[a]], sub, axes=(1, a)), 0, a)
    grids = np.meshgrid(*supports, indexing="ij")
    order = np.argsort(take(sub.size), kind="stable")
    idx = np.stack([g.ravel() for g in grids])[:, order].astype(np.int32)
    val = sub.ravel()[order].astype(np.float64)
    return CooTensor(tuple(dims), idx, val), G, factors
