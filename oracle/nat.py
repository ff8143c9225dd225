"""FP64 reference of the neural acoustic transfer (NAT) field's forward pass (paper Sec. 3.3 and
3.4): grid encoding + positional encoding + MLP.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the tests, the smoke check and the bench's
CPU leg use it; the product library never does. It shares no code with the CUDA path.

The network, as this build reads the paper (Sec. 3.3, Eq. 3 and 4; Sec. 3.4):
  * inputs: x = (theta/pi, phi/(2 pi), (r - r_lo)/(r_hi - r_lo), v_1..v_c, f), each in [0, 1]:
    the listener's spherical coordinates, then the condition variables and the frequency;
  * multi-resolution grid G over (x_0, x_1, x_2): 4 levels of N_l = 8, 16, 32, 64 cells per
    axis, 4 features per vertex, trilinear interpolation of the 8 surrounding vertices; a level
    with (N_l + 1)^3 <= T vertices is stored densely, a finer one through the spatial hash of
    Mueller et al. (2022), (i * 1) xor (j * 2654435761) xor (k * 805459861) mod T;
  * positional encoding P of the condition variables and the frequency only (x_3 onwards):
    sin(2^l pi x_d), cos(2^l pi x_d), l = 0..5;
  * MLP on [G, P(v), P(f)] (zero-padded to 128): four 128-wide layers with ReLU, then a linear
    layer to the outputs (Sec. 3.4).
The grid tables are held in half precision, as tiny-cuda-nn (the paper's implementation, Sec. 3.4)
stores its grid parameters: `encode` rounds them to FP16 first, like the library does when a
field is created. The GPU kernel feeds the tensor cores BF16 activations and weights with FP32 accumulation; this
reference takes the same BF16 weights and rounds every layer's input to BF16 the same way, and
computes everything else in FP64.
"""
from __future__ import annotations

import numpy as np

LEVELS = (8, 16, 32, 64)
FEATURES = 4
PE_FREQS = 6
WIDTH = 128
HIDDEN = 4
PRIMES = (1, 2654435761, 805459861)


def to_bf16(a):
    """Round float64/float32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a):
    """The BF16 bit patterns (uint16) of values that are already BF16-representable."""
    f = np.asarray(a, dtype=np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def level_size(N, table_log2):
    return min((N + 1) ** 3, 1 << table_log2)


def level_index(i, j, k, N, table_log2):
    """Table row of grid vertex (i, j, k) of a level with N cells per axis."""
    T = 1 << table_log2
    if (N + 1) ** 3 <= T:
        return (i + (N + 1) * (j + (N + 1) * k)).astype(np.int64)
    h = (i.astype(np.uint64) * np.uint64(PRIMES[0])) ^ (j.astype(np.uint64) * np.uint64(PRIMES[1])) \
        ^ (k.astype(np.uint64) * np.uint64(PRIMES[2]))
    return (h & np.uint64(0xFFFFFFFF)).astype(np.int64) % T


def grid_features(x3, tables, table_log2):
    """x3: (n, 3) in [0, 1]; tables: list of (rows, 4) arrays. Returns (n, 16)."""
    out = []
    for lvl, N in enumerate(LEVELS):
        p = np.clip(x3, 0.0, 1.0) * N
        i0 = np.minimum(np.floor(p).astype(np.int64), N - 1)
        w = p - i0
        f = np.zeros((x3.shape[0], FEATURES))
        for c in range(8):
            d = np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1])
            wt = np.prod(np.where(d == 1, w, 1.0 - w), axis=1)
            idx = level_index(i0[:, 0] + d[0], i0[:, 1] + d[1], i0[:, 2] + d[2], N, table_log2)
            f += wt[:, None] * tables[lvl][idx]
        out.append(f)
    return np.concatenate(out, axis=1)


def positional(x):
    """(n, D) -> (n, 12 D): for each input, sin then cos of 2^l pi x, l = 0..5."""
    cols = []
    for d in range(x.shape[1]):
        for l in range(PE_FREQS):
            a = (2.0 ** l) * np.pi * x[:, d]
            cols.append(np.sin(a))
            cols.append(np.cos(a))
    return np.stack(cols, axis=1)


def to_half(a):
    """Round to the nearest FP16 value (ties to even) through FP32, returned as float64: the
    grid tables' storage precision."""
    return np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float64)


def encode(x, tables, table_log2):
    """The 128-wide MLP input: 16 grid features of (x_0, x_1, x_2) from the half-precision
    tables, the positional encoding of x_3 onwards (v, then f), zeros."""
    tables = [to_half(t) for t in tables]
    e = np.concatenate([grid_features(x[:, :3], tables, table_log2), positional(x[:, 3:])], axis=1)
    if e.shape[1] > WIDTH:
        raise ValueError("too many inputs for a 128-wide first layer")
    return np.pad(e, ((0, 0), (0, WIDTH - e.shape[1])))


def forward(x, tables, weights, biases, table_log2):
    """x: (n, D) in [0, 1]. weights: 5 arrays (out, in) of BF16-representable values (four
    128 x 128, then n_out x 128); biases: 5 arrays. Returns (n, n_out)."""
    h = to_bf16(encode(np.asarray(x, dtype=np.float64), tables, table_log2))
    for l in range(HIDDEN):
        h = to_bf16(np.maximum(h @ weights[l].T + biases[l], 0.0))
    return h @ weights[HIDDEN].T + biases[HIDDEN]


def random_model(n_cond=2, n_out=8, table_log2=18, seed=0):
    """Seeded random parameters of the shapes above (BF16 weights, FP32 tables and biases)."""
    rng = np.random.default_rng(seed)
    tables = [to_half(rng.uniform(-1.0, 1.0, size=(level_size(N, table_log2), FEATURES))) for N in LEVELS]
    weights, biases = [], []
    for l in range(HIDDEN + 1):
        n_o = n_out if l == HIDDEN else WIDTH
        weights.append(to_bf16(rng.normal(0.0, np.sqrt(2.0 / WIDTH), size=(n_o, WIDTH))))
        biases.append(rng.normal(0.0, 0.05, size=n_o).astype(np.float32).astype(np.float64))
    return dict(n_cond=n_cond, n_out=n_out, table_log2=table_log2, tables=tables, weights=weights,
                biases=biases)
