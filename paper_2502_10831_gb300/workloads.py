"""Seeded synthetic angle workloads (inputs only; none of the method's arithmetic).

Both the CUDA library's tests/benchmark and the FP64 oracle are fed from here.
The paper benchmarks on 1000 angles drawn uniformly from [-1e6, 1e6] with seed
2024873 (Sec. 4); its RNG is not named, so every workload below uses numpy's
PCG64 seeded from that number, with one SeedSequence stream per (workload,
chunk) so that large arrays are generated chunk-parallel and any chunk can be
regenerated on its own.

Mixtures pick a component per element (categorical draw), which gives the
stated fractions in expectation without a global permutation.

  parity     2^20 f32: 90% U[-2pi, 2pi], 10% within 1e-3 of +-pi/2, +-3pi/2
  bandwidth  2^28 f32: 80% U[-100pi, 100pi], 10% within 1e-4 of k pi/12
             (|k| <= 1200), 10% within 1e-3 of odd multiples of pi/2
  half       the bandwidth mixture stored as fp16 (uniform part U[-60, 60],
             nodes and poles kept where |x| <= 60) or bf16
  large      2^24 f32, |x| log-uniform in [1, 1e5], random sign
  batch      4096 arrays, lengths floor(exp U[ln 100, ln 1e6]), values
             U[-8pi, 8pi], selector uniform over sin/cos/tan/sincos
  autograd   [8192, 4096] f32 U[-4pi, 4pi]; w, v, u ~ N(0, 1)
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

SEED = 2024873
PI = math.pi

# workload ids used in the seed sequence
_WL = {"parity": 1, "bandwidth": 2, "half16": 3, "half_bf16": 4, "large": 5,
       "batch": 6, "autograd": 7, "edge": 8, "paper": 9}

CHUNK = 1 << 22


def _rng(workload: str, *idx: int, seed: int = SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, _WL[workload], *idx])))


def _mixture(rng: np.random.Generator, m: int, lim: float, p_uniform: float, p_node: float,
             node_kmax: int, node_off: float, pole_off: float) -> np.ndarray:
    """Per-element mixture of uniform, near-node and near-pole angles (float64)."""
    comp = rng.random(m)
    uni = rng.uniform(-lim, lim, m)
    k = rng.integers(-node_kmax, node_kmax + 1, m)
    node = k * (PI / 12.0) + rng.uniform(-node_off, node_off, m)
    # odd multiples (2j+1) pi/2 that lie inside [-lim, lim]
    jmax = int(math.floor((lim / (PI / 2.0) - 1.0) / 2.0))
    j = rng.integers(-jmax - 1, jmax + 1, m)
    pole = (2 * j + 1) * (PI / 2.0) + rng.uniform(-pole_off, pole_off, m)
    out = np.where(comp < p_uniform, uni, np.where(comp < p_uniform + p_node, node, pole))
    return out


def _chunked(n: int, fn, dtype, threads: int | None = None) -> np.ndarray:
    out = np.empty(n, dtype=dtype)
    nchunks = (n + CHUNK - 1) // CHUNK

    def work(c):
        lo = c * CHUNK
        hi = min(n, lo + CHUNK)
        out[lo:hi] = fn(c, hi - lo)

    if nchunks <= 1:
        for c in range(nchunks):
            work(c)
    else:
        with ThreadPoolExecutor(max_workers=threads or 16) as ex:
            list(ex.map(work, range(nchunks)))
    return out


def parity(n: int = 1 << 20, seed: int = SEED) -> np.ndarray:
    """90% U[-2pi, 2pi], 10% within 1e-3 of the four poles +-pi/2, +-3pi/2 (f32)."""
    def gen(c, m):
        r = _rng("parity", c, seed=seed)
        return _mixture(r, m, 2 * PI, 0.9, 0.0, 0, 0.0, 1e-3).astype(np.float32)
    return _chunked(n, gen, np.float32)


def bandwidth(n: int = 1 << 28, seed: int = SEED) -> np.ndarray:
    """80% U[-100pi, 100pi], 10% near k pi/12 (|k|<=1200, +-1e-4), 10% near poles (+-1e-3)."""
    def gen(c, m):
        r = _rng("bandwidth", c, seed=seed)
        return _mixture(r, m, 100 * PI, 0.8, 0.1, 1200, 1e-4, 1e-3).astype(np.float32)
    return _chunked(n, gen, np.float32)


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest-even) and return the 16-bit patterns."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = np.isnan(x)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
    r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def half16(n: int = 1 << 28, seed: int = SEED) -> np.ndarray:
    """Bandwidth mixture for fp16: uniform part U[-60, 60], nodes/poles with |x| <= 60.
    Returns float16 values."""
    def gen(c, m):
        r = _rng("half16", c, seed=seed)
        return _mixture(r, m, 60.0, 0.8, 0.1, int(60.0 // (PI / 12.0)), 1e-4, 1e-3).astype(np.float16)
    return _chunked(n, gen, np.float16)


def half_bf16(n: int = 1 << 28, seed: int = SEED) -> np.ndarray:
    """Bandwidth mixture rounded to bfloat16; returns uint16 bit patterns."""
    def gen(c, m):
        r = _rng("half_bf16", c, seed=seed)
        v = _mixture(r, m, 100 * PI, 0.8, 0.1, 1200, 1e-4, 1e-3).astype(np.float32)
        return f32_to_bf16_bits(v)
    return _chunked(n, gen, np.uint16)


def large(n: int = 1 << 24, seed: int = SEED) -> np.ndarray:
    """|x| log-uniform in [1, 1e5] with random sign (f32)."""
    def gen(c, m):
        r = _rng("large", c, seed=seed)
        mag = np.exp(r.uniform(0.0, math.log(1e5), m))
        sgn = np.where(r.random(m) < 0.5, -1.0, 1.0)
        return (sgn * mag).astype(np.float32)
    return _chunked(n, gen, np.float32)


BATCH_FUNCS = ("sin", "cos", "tan", "sincos")


def batch_spec(count: int = 4096, lo: int = 100, hi: int = 1_000_000, seed: int = SEED):
    """Lengths floor(exp U[ln lo, ln hi]) and selectors uniform over sin/cos/tan/sincos."""
    r = _rng("batch", 0, seed=seed)
    lengths = np.floor(np.exp(r.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    sel = r.integers(0, 4, count)
    return lengths, sel


def batch_array(i: int, length: int, seed: int = SEED) -> np.ndarray:
    """Values of array i of the ragged batch: U[-8pi, 8pi] (f32)."""
    r = _rng("batch", 1 + i, seed=seed)
    return r.uniform(-8 * PI, 8 * PI, int(length)).astype(np.float32)


def autograd(shape=(8192, 4096), seed: int = SEED):
    """x ~ U[-4pi, 4pi]; w, v, u ~ N(0, 1); all f32 of the same shape."""
    n = int(np.prod(shape))

    def gen_of(k, kind):
        def gen(c, m):
            r = _rng("autograd", k, c, seed=seed)
            if kind == "x":
                return r.uniform(-4 * PI, 4 * PI, m).astype(np.float32)
            return r.standard_normal(m).astype(np.float32)
        return gen

    x = _chunked(n, gen_of(0, "x"), np.float32).reshape(shape)
    w = _chunked(n, gen_of(1, "n"), np.float32).reshape(shape)
    v = _chunked(n, gen_of(2, "n"), np.float32).reshape(shape)
    u = _chunked(n, gen_of(3, "n"), np.float32).reshape(shape)
    return x, w, v, u


def paper_angles(num: int = 1000, seed: int = SEED) -> np.ndarray:
    """num angles U[-1e6, 1e6] in double, as in the paper's benchmark (Sec. 4)."""
    return _rng("paper", 0, seed=seed).uniform(-1e6, 1e6, num)


def away_from_nodes(x: np.ndarray, margin: float = 1e-3) -> np.ndarray:
    """Boolean mask of angles at least `margin` from every k pi/12 (nodes and poles)."""
    step = PI / 12.0
    xd = np.asarray(x, dtype=np.float64)
    d = np.abs(xd - np.round(xd / step) * step)
    return d >= margin


def edge_values() -> np.ndarray:
    """Hand-picked f32 inputs: signed zeros, tiny and subnormal values, values
    next to pi/12 nodes and odd multiples of pi/2, the fast/slow reduction
    boundary, very large magnitudes, infinities and NaN."""
    f = np.float32
    vals = [0.0, -0.0, 1e-45, -1e-45, 1e-38, 1e-30, -1e-10, 1e-7, 0.5, -0.5, 1.0, -1.0]
    for k in range(-48, 49):
        c = f(k * PI / 12.0)
        vals += [c, np.nextafter(c, f(np.inf)), np.nextafter(c, f(-np.inf))]
    for j in (1, 3, 5, 7, 101, 199, 2047, 2049, 65535):
        c = f(j * PI / 2.0)
        vals += [c, -c, np.nextafter(c, f(np.inf)), np.nextafter(c, f(-np.inf))]
    for b in (f(1024.0 * PI), f(2.0 ** 20), f(2.0 ** 31)):
        vals += [b, -b, np.nextafter(b, f(0.0)), np.nextafter(b, f(np.inf))]
    vals += [1e5, -1e5, 1e6, 3.0e9, -6.7e9, 1e10, 2.0 ** 40, 1e20, -1e30, 3.4e38, -3.4e38]
    vals += [np.inf, -np.inf, np.nan]
    return np.array(vals, dtype=np.float32)
