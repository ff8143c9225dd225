"""Pins of the NAT-field reference forward pass (paper Sec. 3.3, 3.4). CPU only."""
import numpy as np

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
    m = nat.random_model(n_cond=1, n_out=3, table_log2=12, seed=3)
    W = [np.eye(128) for _ in range(4)] + [np.zeros((3, 128))]
    W[4][0, 16] = 1.0   # the first positional feature: sin(pi x_3)
    W[4][2, 0] = 2.0    # twice the first grid feature
    bias = [np.zeros(128)] * 4 + [np.array([0.0, 0.75, 0.0])]
    x = np.random.default_rng(1).random((64, 5))
    out = nat.forward(x, m["tables"], W, bias, 12)
    enc = nat.to_bf16(nat.encode(x, m["tables"], 12))
    assert np.allclose(out[:, 0], np.maximum(enc[:, 16], 0.0))
    assert np.allclose(enc[:, 16], nat.to_bf16(np.sin(np.pi * x[:, 3])))
    assert np.allclose(enc[:, 16 + 12 * 2:], 0.0)  # two encoded inputs (v_1, f), then padding
    assert np.allclose(out[:, 1], 0.75)
    assert np.allclose(out[:, 2], 2.0 * np.maximum(enc[:, 0], 0.0))


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


def test_hidden_layers_apply_relu_and_round():
    """A hidden layer of -identity zeroes every positive encoded input (ReLU), and the output
    layer sees BF16-rounded activations (a bias of 2^-12 added to 1 is lost)."""
    m = nat.random_model(n_cond=0, n_out=2, table_log2=12, seed=7)
    W = [-np.eye(128), -np.eye(128), np.eye(128), np.eye(128), np.zeros((2, 128))]
    W[4][0, :] = 1.0
    W[4][1, 20] = 1.0
    bias = [np.zeros(128), np.zeros(128), np.full(128, 1.0), np.full(128, 2.0 ** -12), np.zeros(2)]
    x = np.random.default_rng(2).random((32, 4))
    enc = nat.to_bf16(nat.encode(x, m["tables"], 12))
    out = nat.forward(x, m["tables"], W, bias, 12)
    # after two -I layers: relu(-relu(-e)) = 0 for every e, then relu(0 + 1) = 1, then 1 + 2^-12 -> 1
    assert np.allclose(out[:, 0], 128.0) and np.allclose(out[:, 1], 1.0)
    assert enc.shape == (32, 128)


def test_tables_are_rounded_to_half():
    """Table values are used at FP16 precision: a value between two FP16 numbers moves to the
    nearest, and the encoding of a query on a vertex returns the rounded value."""
    assert nat.to_half(1.0 + 2.0 ** -12)[()] == 1.0 and nat.to_half(1.0 + 3 * 2.0 ** -11)[()] == 1.0 + 2.0 ** -9
    log2 = 12
    tables = [np.full((nat.level_size(N, log2), 4), 1.0 + 2.0 ** -12) for N in nat.LEVELS]
    e = nat.encode(np.array([[0.0, 0.0, 0.0, 0.5]]), tables, log2)
    assert np.all(e[0, :16] == 1.0)
