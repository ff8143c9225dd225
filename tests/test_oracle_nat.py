"""Pins of the NAT-field reference forward pass (paper Sec. 3.3, 3.4) and of its rounding-error
model. CPU only."""
import numpy as np

import synthetic as S
from oracle import nat


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, -2.5, 1e-3])
    r = nat.to_bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -7 and r[3] == -2.5  # ties to even
    assert abs(r[4] - 1e-3) <= 2.0 ** -9 * 1e-3
    assert np.all(nat.to_bf16(r) == r)


def test_trilinear_grid_reproduces_linear_data():
    """Dense levels hold a linear function of the vertex coordinates: the interpolated feature
    equals that function at the query point (pins the vertex indexing and the weights)."""
    rng = np.random.default_rng(0)
    log2 = 18
    a = rng.normal(size=(4, 3))
    b = rng.normal(size=4)
    tables = []
    for N in nat.LEVELS:
        rows = nat.level_size(N, log2)
        t = np.zeros((rows, 4))
        if (N + 1) ** 3 <= (1 << log2):
            i, j, k = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
            i, j, k = i.ravel(), j.ravel(), k.ravel()
            idx = nat.level_index(i, j, k, N, log2)
            t[idx] = (np.stack([i, j, k], 1) / N) @ a.T + b
        tables.append(t)
    x = rng.random((500, 3))
    x[:5] = [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.999999, 0.5, 0], [0.125, 0.25, 0.375]]
    f = nat.grid_features(x, tables, log2)
    expect = x @ a.T + b
    for lvl, N in enumerate(nat.LEVELS[:3]):  # the dense levels
        assert np.allclose(f[:, 4 * lvl:4 * lvl + 4], expect, atol=1e-12)


def test_hashed_level_uses_the_whole_table():
    log2 = 14
    N = nat.LEVELS[-1]
    i, j, k = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
    idx = nat.level_index(i.ravel(), j.ravel(), k.ravel(), N, log2)
    assert idx.min() >= 0 and idx.max() < (1 << log2)
    counts = np.bincount(idx, minlength=1 << log2)
    assert np.mean(counts > 0) > 0.95 and counts.max() < 4 * (N + 1) ** 3 / (1 << log2)


def test_positional_encoding_values():
    x = np.array([[0.5, 0.25]])
    pe = nat.positional(x)
    assert pe.shape == (1, 24)
    assert np.isclose(pe[0, 0], 1.0) and np.isclose(pe[0, 1], 0.0)       # sin, cos(pi/2)
    assert np.isclose(pe[0, 12], np.sin(np.pi / 4)) and np.isclose(pe[0, 13], np.cos(np.pi / 4))
    assert np.allclose(pe[:, 0::2] ** 2 + pe[:, 1::2] ** 2, 1.0)


def test_mlp_layer_order_and_transposes():
    """Identity hidden layers and a one-hot output layer pass one encoded input through."""
    m = S.nat_params(n_cond=1, n_out=3, table_log2=12, seed=3)
    W = [np.eye(128) for _ in range(4)] + [np.zeros((3, 128))]
    W[4][0, 16] = 1.0   # the first positional feature: sin(pi x_3)
    W[4][2, 0] = 2.0    # twice the first grid feature
    bias = [np.zeros(128)] * 4 + [np.array([0.0, 0.75, 0.0])]
    x = np.random.default_rng(1).random((64, 5))
    out = nat.forward(x, m["tables"], W, bias, 12)
    enc = nat.encode(x, m["tables"], 12)
    assert np.allclose(out[:, 0], np.maximum(enc[:, 16], 0.0), rtol=0, atol=1e-15)
    assert np.allclose(enc[:, 16], np.sin(np.pi * x[:, 3]), rtol=0, atol=1e-15)
    assert np.allclose(enc[:, 16 + 12 * 2:], 0.0)  # two encoded inputs (v_1, f), then padding
    assert np.allclose(out[:, 1], 0.75)
    assert np.allclose(out[:, 2], 2.0 * np.maximum(enc[:, 0], 0.0), rtol=0, atol=1e-15)


def test_hash_is_the_published_spatial_hash():
    """The hashed rows follow the spatial hash of Mueller et al. (2022) evaluated with Python's
    unbounded integers and an explicit 32-bit wrap: xor of coordinate x prime, modulo T."""
    rng = np.random.default_rng(5)
    ijk = rng.integers(0, 65, size=(200, 3))
    for log2 in (12, 18):
        got = nat.level_index(ijk[:, 0], ijk[:, 1], ijk[:, 2], 64, log2)
        for (i, j, k), g in zip(ijk, got):
            h = ((int(i) * 1) ^ (int(j) * 2654435761) ^ (int(k) * 805459861)) % (1 << 32)
            assert g == h % (1 << log2)


def test_hidden_layers_apply_relu_and_the_rounded_model_rounds():
    """A hidden layer of -identity zeroes every positive encoded input (ReLU) in both forms; the
    bit-level model also rounds the activations to BF16 (a bias of 2^-12 added to 1 is lost),
    the FP64 network keeps it."""
    m = S.nat_params(n_cond=0, n_out=2, table_log2=12, seed=7)
    W = [-np.eye(128), -np.eye(128), np.eye(128), np.eye(128), np.zeros((2, 128))]
    W[4][0, :] = 1.0
    W[4][1, 20] = 1.0
    bias = [np.zeros(128), np.zeros(128), np.full(128, 1.0), np.full(128, 2.0 ** -12), np.zeros(2)]
    x = np.random.default_rng(2).random((32, 4))
    # after two -I layers: relu(-relu(-e)) = 0 for every e, then relu(0 + 1) = 1, then 1 + 2^-12
    out = nat.forward_rounded(x, m["tables"], W, bias, 12)
    assert np.allclose(out[:, 0], 128.0) and np.allclose(out[:, 1], 1.0)
    exact = nat.forward(x, m["tables"], W, bias, 12)
    assert np.allclose(exact[:, 0], 128.0 * (1.0 + 2.0 ** -12)) and np.allclose(exact[:, 1], 1.0 + 2.0 ** -12)


def test_tables_are_rounded_to_half():
    """Table values are used at FP16 precision: a value between two FP16 numbers moves to the
    nearest, and the encoding of a query on a vertex returns the rounded value."""
    assert nat.to_half(1.0 + 2.0 ** -12)[()] == 1.0 and nat.to_half(1.0 + 3 * 2.0 ** -11)[()] == 1.0 + 2.0 ** -9
    log2 = 12
    tables = [np.full((nat.level_size(N, log2), 4), 1.0 + 2.0 ** -12) for N in nat.LEVELS]
    x = np.array([[0.0, 0.0, 0.0, 0.5]])
    W = [np.eye(128) for _ in range(4)] + [np.eye(128)[:16]]
    b = [np.zeros(128)] * 4 + [np.zeros(16)]
    assert np.all(nat.forward_rounded(x, tables, W, b, log2)[0] == 1.0)
    assert np.all(nat.forward(x, tables, W, b, log2)[0] == 1.0 + 2.0 ** -12)  # FP64: unrounded


def _perturbed_forward(x, m, rng, u_t, u_w, u_in):
    """The network with every stored value v replaced by v (1 + d), d uniform in [-u, u] and
    independent: tables (u_t), weights (u_w), each layer's input (u_in). FP64 otherwise."""
    rel = lambda a, u: a * (1.0 + rng.uniform(-u, u, size=np.shape(a)))
    tables = [rel(np.asarray(t, np.float64), u_t) for t in m["tables"]]
    W = [rel(np.asarray(w, np.float64), u_w) for w in m["weights"]]
    b = [np.asarray(v, np.float64) for v in m["biases"]]
    h = rel(nat.encode(x, tables, m["table_log2"]), u_in)
    for l in range(4):
        h = rel(np.maximum(h @ W[l].T + b[l], 0.0), u_in)
    return h @ W[4].T + b[4]


def test_rounding_sigma_matches_monte_carlo():
    """The first-order propagation in rounding_sigma against brute force: 400 forward passes
    with independent uniform relative perturbations of exactly the modelled size (variance
    u^2 v^2 / 3 per stored value) give, per output, an empirical standard deviation that the
    formula must reproduce. A dropped ReLU mask, a transposed weight or a missing source shifts
    the ratio far outside the band."""
    m = S.nat_params(n_cond=2, n_out=3, table_log2=14, seed=21)
    x = S.nat_queries(40, 6, 22).astype(np.float64)
    args = (m["tables"], m["weights"], m["biases"], m["table_log2"])
    ref = nat.forward(x, *args)
    rng = np.random.default_rng(23)
    for u_t, u_w, u_in in ((0.0, 2.0 ** -8, 0.0), (0.0, 0.0, 2.0 ** -8), (2.0 ** -6, 0.0, 0.0),
                           (2.0 ** -11, 2.0 ** -8, 2.0 ** -8)):
        dev = np.stack([_perturbed_forward(x, m, rng, u_t, u_w, u_in) - ref for _ in range(400)])
        emp = np.sqrt(np.mean(dev ** 2, axis=0))
        sig = nat.rounding_sigma(x, *args, u_table=u_t, u_weight=u_w, u_input=u_in, u_acc=0.0)
        ratio = emp / sig
        if u_t > 0 and u_w == 0:
            # table corners are modelled as fully correlated (an upper estimate)
            assert np.all(ratio <= 1.15) and np.median(ratio) > 0.4, (np.median(ratio), ratio.max())
        else:
            assert 0.9 < np.median(ratio) < 1.1 and np.all((ratio > 0.6) & (ratio < 1.4)), \
                (u_t, u_w, u_in, np.median(ratio), ratio.min(), ratio.max())


def test_rounded_model_within_the_derived_bound():
    """The literal roundings (FP16 tables, BF16 weights and layer inputs) stay within the bound
    that the GPU parity test applies: every output within 12 sigma, mean (dev / sigma)^2 <= 1.5."""
    for nc, no, lg, seed in ((2, 8, 18, 1), (0, 1, 12, 3), (5, 33, 20, 4)):
        m = S.nat_params(n_cond=nc, n_out=no, table_log2=lg, seed=seed)
        x = S.nat_queries(1500, 4 + nc, seed).astype(np.float64)
        args = (m["tables"], m["weights"], m["biases"], lg)
        d = np.abs(nat.forward_rounded(x, *args) - nat.forward(x, *args)) / nat.rounding_sigma(x, *args)
        assert d.max() <= 12.0 and np.mean(d ** 2) <= 1.5, (d.max(), np.mean(d ** 2))
        assert np.mean(d ** 2) > 0.1  # the model is not vacuous either
