"""FP64 reference of the neural acoustic transfer (NAT) field's forward pass (paper Sec. 3.3 and
3.4): grid encoding + positional encoding + MLP.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the tests, the smoke check and the bench's
CPU leg use it; the product library never does. It shares no code with the CUDA path, and the
parameters it is given come from the seeded generator in synthetic/ (plain float32 draws).

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

`forward` is that network in FP64 with the parameters exactly as given: no rounding anywhere.
The paper runs the network in reduced precision (tiny-cuda-nn, Sec. 3.4), and a fast kernel
stores its parameters and layer inputs in reduced precision too, so its outputs differ from
`forward` by rounding. `rounding_sigma` states how much, from first principles: the first-order
propagation through the network of independent round-to-nearest errors in each stored value
(a standard probabilistic rounding-error model), for storage precisions given as unit
roundoffs. `forward_rounded` applies such roundings literally (FP16 tables, BF16 weights and
layer inputs) and is only a second, bit-level model for tests.
"""
from __future__ import annotations

import numpy as np

LEVELS = (8, 16, 32, 64)
FEATURES = 4
PE_FREQS = 6
WIDTH = 128
HIDDEN = 4
PRIMES = (1, 2654435761, 805459861)

U_BF16 = 2.0 ** -8   # unit roundoff of BF16 (8 significant bits), round to nearest
U_FP16 = 2.0 ** -11  # unit roundoff of IEEE half precision (11 significant bits)
U_FP32 = 2.0 ** -24  # unit roundoff of IEEE single precision (24 significant bits)


def to_bf16(a):
    """Round float64/float32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def to_half(a):
    """Round to the nearest FP16 value (ties to even) through FP32, returned as float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float64)


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


def _grid(x3, tables, table_log2):
    """Trilinear features (n, 16) and, per feature, the sum over the 8 corners of |w T|."""
    out, mag = [], []
    for lvl, N in enumerate(LEVELS):
        t = np.asarray(tables[lvl], dtype=np.float64)
        p = np.clip(x3, 0.0, 1.0) * N
        i0 = np.minimum(np.floor(p).astype(np.int64), N - 1)
        w = p - i0
        f = np.zeros((x3.shape[0], FEATURES))
        a = np.zeros((x3.shape[0], FEATURES))
        for c in range(8):
            d = np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1])
            wt = np.prod(np.where(d == 1, w, 1.0 - w), axis=1)
            idx = level_index(i0[:, 0] + d[0], i0[:, 1] + d[1], i0[:, 2] + d[2], N, table_log2)
            f += wt[:, None] * t[idx]
            a += np.abs(wt[:, None] * t[idx])
        out.append(f)
        mag.append(a)
    return np.concatenate(out, axis=1), np.concatenate(mag, axis=1)


def grid_features(x3, tables, table_log2):
    """x3: (n, 3) in [0, 1]; tables: list of (rows, 4) arrays. Returns (n, 16)."""
    return _grid(x3, tables, table_log2)[0]


def positional(x):
    """(n, D) -> (n, 12 D): for each input, sin then cos of 2^l pi x, l = 0..5."""
    cols = []
    for d in range(x.shape[1]):
        for l in range(PE_FREQS):
            a = (2.0 ** l) * np.pi * x[:, d]
            cols.append(np.sin(a))
            cols.append(np.cos(a))
    return np.stack(cols, axis=1)


def encode(x, tables, table_log2):
    """The 128-wide MLP input: 16 grid features of (x_0, x_1, x_2), the positional encoding of
    x_3 onwards (v, then f), zeros."""
    x = np.asarray(x, dtype=np.float64)
    e = np.concatenate([grid_features(x[:, :3], tables, table_log2), positional(x[:, 3:])], axis=1)
    if e.shape[1] > WIDTH:
        raise ValueError("too many inputs for a 128-wide first layer")
    return np.pad(e, ((0, 0), (0, WIDTH - e.shape[1])))


def forward(x, tables, weights, biases, table_log2):
    """The network in FP64. x: (n, D) in [0, 1]; tables: 4 arrays (rows, 4); weights: 5 arrays
    (out, in), four 128 x 128 then n_out x 128; biases: 5 arrays. Returns (n, n_out)."""
    h = encode(x, tables, table_log2)
    W = [np.asarray(w, dtype=np.float64) for w in weights]
    b = [np.asarray(v, dtype=np.float64) for v in biases]
    for l in range(HIDDEN):
        h = np.maximum(h @ W[l].T + b[l], 0.0)
    return h @ W[HIDDEN].T + b[HIDDEN]


def rounding_sigma(x, tables, weights, biases, table_log2, u_table=U_FP16, u_weight=U_BF16,
                   u_input=U_BF16, u_acc=U_FP32):
    """Standard deviation, per output (n, n_out), of the deviation of a forward pass that stores
    the grid tables with unit roundoff u_table, the weights with u_weight and every layer's
    input (the encoding, each hidden activation) with u_input, and accumulates with u_acc.

    Model (probabilistic rounding-error analysis): rounding a value v to nearest leaves an
    error of at most u |v| (half a unit in the last place), taken as independent, zero-mean
    and uniform, so of variance at most u^2 v^2 / 3. To first order the output deviation is
    sum_s J_s e_s over the rounding errors e_s with J_s = d y / d(value s), so its variance is
    sum_s J_s^2 Var(e_s). With h_l the input of layer l, z_l = W_l h_l + b_l, D_l the ReLU mask
    and y = z_4:
      d y / d z_4 = I,  d y / d h_l = (d y / d z_l) W_l,  d y / d z_l = (d y / d h_{l+1}) D_l;
      input rounding   sum_k (dy/dh_l)_k^2  u_input^2 h_lk^2 / 3,          l = 0..4;
      weight rounding  sum_j (dy/dz_l)_j^2  u_weight^2 (W_l^2 h_l^2)_j / 3, l = 0..4;
      accumulation     sum_j (dy/dz_l)_j^2  128 u_acc^2 ((|W_l| |h_l|)_j)^2 / 3;
      table rounding   sum_c (dy/dh_0)_c^2  u_table^2 (sum_corners |w T|)_c^2 / 3 over the 16
                       grid features (corners taken as fully correlated: an upper estimate).
    By Hoeffding's inequality a sum of independent zero-mean terms bounded by a_s exceeds t
    with probability at most 2 exp(-t^2 / (2 sum a_s^2)); with |e_s| <= sqrt(3) sigma_s that is
    2 exp(-t^2 / (6 sigma^2)), so |deviation| <= 12 sigma fails with probability < 1e-10."""
    x = np.asarray(x, dtype=np.float64)
    g, gmag = _grid(x[:, :3], tables, table_log2)
    h0 = np.concatenate([g, positional(x[:, 3:])], axis=1)
    h0 = np.pad(h0, ((0, 0), (0, WIDTH - h0.shape[1])))
    W = [np.asarray(w, dtype=np.float64) for w in weights]
    b = [np.asarray(v, dtype=np.float64) for v in biases]
    hs, masks = [h0], []
    for l in range(HIDDEN):
        z = hs[-1] @ W[l].T + b[l]
        masks.append((z > 0.0).astype(np.float64))
        hs.append(np.maximum(z, 0.0))
    n, n_out = x.shape[0], W[HIDDEN].shape[0]
    var = np.zeros((n, n_out))
    dz = np.broadcast_to(np.eye(n_out), (n, n_out, n_out))  # d y / d z_4
    for l in range(HIDDEN, -1, -1):
        h = hs[l]
        wh2 = (h ** 2) @ (W[l] ** 2).T                        # (W_l^2 h_l^2)_j
        acc = (np.abs(h) @ np.abs(W[l]).T) ** 2               # ((|W_l| |h_l|)_j)^2
        dz2 = dz ** 2
        var += np.einsum("noj,nj->no", dz2, wh2) * (u_weight ** 2 / 3.0)
        var += np.einsum("noj,nj->no", dz2, acc) * (WIDTH * u_acc ** 2 / 3.0)
        dh = np.einsum("noj,jk->nok", dz, W[l])               # d y / d h_l
        var += np.einsum("nok,nk->no", dh ** 2, h ** 2) * (u_input ** 2 / 3.0)
        if l == 0:
            var += np.einsum("nok,nk->no", dh[:, :, :16] ** 2, gmag ** 2) * (u_table ** 2 / 3.0)
        else:
            dz = dh * masks[l - 1][:, None, :]                # d y / d z_{l-1}
    return np.sqrt(var)


def forward_rounded(x, tables, weights, biases, table_log2):
    """A bit-level model of reduced-precision storage, for a second, tighter test: tables
    rounded to FP16, weights to BF16, the encoding and every hidden activation rounded to BF16
    (after the ReLU), everything else in FP64."""
    tables = [to_half(t) for t in tables]
    h = to_bf16(encode(x, tables, table_log2))
    W = [to_bf16(w) for w in weights]
    b = [np.asarray(v, dtype=np.float64) for v in biases]
    for l in range(HIDDEN):
        h = to_bf16(np.maximum(h @ W[l].T + b[l], 0.0))
    return h @ W[HIDDEN].T + b[HIDDEN]
