"""GPU parity of the neural acoustic transfer field's forward pass (paper Sec. 3.3 and 3.4:
grid encoding, positional encoding, 4 x 128 MLP) against the FP64 oracle.

Parameters come from synthetic.nat_params (plain float32 draws); the library rounds the tables
to FP16 and the weights to BF16 itself, and feeds the tensor cores BF16 layer inputs. The oracle
runs the network in FP64 on the unrounded parameters, so the two differ by the rounding of the
stored values. The bound is derived, per output, from those storage precisions (unit roundoff
2^-11 for the FP16 tables, 2^-8 for the BF16 weights and layer inputs, 2^-24 for the FP32
accumulation): oracle.nat.rounding_sigma gives the standard deviation sigma of the first-order
rounding error under the usual model of independent round-to-nearest errors, and Hoeffding's
inequality bounds a deviation beyond 12 sigma by a probability below 1e-10 per output. So:
  * every output: |kernel - oracle| <= 12 sigma (+ 1e-6 of the outputs' RMS for FP32 effects
    the model leaves out, such as the FP32 sine and cosine of the positional encoding);
  * with at least 1000 outputs: mean((deviation / sigma)^2) <= 1.5. The model's variances are
    upper estimates (half an ulp is at most u |v|), so this mean is at most 1 in expectation;
    on the CPU a literal rounding model gives about 0.5.
A second, bit-level check compares with oracle.nat.forward_rounded (the same roundings applied
literally in FP64): relative L2 <= 1e-3, the FP32 accumulation moving a value across a BF16
rounding boundary now and then.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
from oracle import nat as O

pytestmark = pytest.mark.gpu

Z_MAX = 12.0
MEAN_Z2 = 1.5
REL_L2_BITS = 1e-3


@pytest.fixture(scope="module")
def nb():
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build
    build.build()
    return nb


def _check(out, x, m):
    out = np.asarray(out, dtype=np.float64)
    args = (m["tables"], m["weights"], m["biases"], m["table_log2"])
    ref = O.forward(x.astype(np.float64), *args)
    sig = O.rounding_sigma(x.astype(np.float64), *args)
    rms = np.sqrt(np.mean(ref ** 2))
    dev = np.abs(out - ref)
    assert np.all(dev <= Z_MAX * sig + 1e-6 * rms), np.max(dev / sig)
    if out.size >= 1000:
        assert np.mean((dev / sig) ** 2) <= MEAN_Z2, np.mean((dev / sig) ** 2)
    bits = O.forward_rounded(x.astype(np.float64), *args)
    rel = np.linalg.norm(out - bits) / np.linalg.norm(bits)
    assert rel <= REL_L2_BITS, rel


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 5000])
def test_forward_matches_oracle(nb, n):
    m = S.nat_params(n_cond=2, n_out=8, table_log2=18, seed=1)
    x = S.nat_queries(n, 6, n)
    with nb.NatField.from_params(m) as f:
        out = f.forward(x)
    assert out.shape == (n, 8)
    _check(out, x, m)


@pytest.mark.parametrize("n_cond,n_out,log2", [(0, 1, 12), (5, 33, 20), (1, 128, 14), (8, 64, 16)])
def test_shapes_and_table_sizes(nb, n_cond, n_out, log2):
    """Hashed levels (2^12: all but the coarsest), all-dense tables (2^20), the widest input
    (D = 12: 8 condition variables), one output and the full 128 outputs."""
    m = S.nat_params(n_cond=n_cond, n_out=n_out, table_log2=log2, seed=2 + n_cond)
    x = S.nat_queries(777, 4 + n_cond, 11)
    with nb.NatField.from_params(m) as f:
        out = f.forward(x)
    _check(out, x, m)


def test_boundary_inputs(nb):
    """Queries on the grid's faces and corners (x = 0 and x = 1 exactly) and on vertex planes."""
    m = S.nat_params(seed=4)
    g = np.array([0.0, 1.0, 0.5, 0.25, 1.0 / 64, 63.0 / 64], np.float32)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = np.concatenate([x, np.tile(np.array([[0.0, 1.0, 0.3]], np.float32), (len(x), 1))], axis=1)
    with nb.NatField.from_params(m) as f:
        out = f.forward(x)
    _check(out, x, m)


def _bf16_torch(a):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _half_torch(a):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.float16).to(torch.float64).numpy()


def test_library_rounds_weights_to_bf16(nb):
    """The field converts the caller's FP32 weights itself. Identity hidden layers pass the first
    positional feature, sin(pi / 2) = 1, through unchanged, so output i is the stored output
    weight W_4[i, 16]: it must equal torch's nearest-even BF16 conversion of the FP32 value."""
    n_out = 64
    rng = np.random.default_rng(7)
    m = S.nat_params(n_cond=1, n_out=n_out, table_log2=12, seed=9)
    W = [np.eye(128, dtype=np.float32) for _ in range(4)] + [np.zeros((n_out, 128), np.float32)]
    col = rng.normal(size=n_out).astype(np.float32)
    col[:8] = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5 + 2.0 ** -10, 1e-3, 3.0e-30, 1.0, 0.0, 65519.0]
    W[4][:, 16] = col
    m["weights"] = W
    m["biases"] = [np.zeros(128, np.float32)] * 4 + [np.zeros(n_out, np.float32)]
    x = np.array([[0.3, 0.6, 0.2, 0.5, 0.5]], np.float32)  # v_1 = 0.5: sin(pi v_1) = 1
    with nb.NatField.from_params(m) as f:
        out = f.forward(x)
    assert np.array_equal(out[0].astype(np.float64), _bf16_torch(col)), (out[0][:8], _bf16_torch(col)[:8])


def test_library_rounds_tables_to_half(nb):
    """The field keeps the tables in FP16. A query on a vertex of the coarsest (dense) level
    reads one table row; values chosen so that FP16 rounding (subnormals below 2^-14, no values
    below 2^-24) and the later BF16 rounding of the layer input both leave a mark that tells
    them apart from BF16 alone. Output = BF16(FP16(t)) exactly."""
    m = S.nat_params(n_cond=0, n_out=4, table_log2=18, seed=10)
    vals = np.array([1.1 * 2.0 ** -20, 3.0e-9, 1.0 + 2.0 ** -11 + 2.0 ** -13, -0.7], np.float32)
    for t in m["tables"]:
        t[:] = 0.0
    m["tables"][0][0, :] = vals                 # vertex (0, 0, 0) of the 8-cell level
    W = [np.eye(128, dtype=np.float32) for _ in range(4)] + [np.zeros((4, 128), np.float32)]
    W[4][np.arange(4), np.arange(4)] = 1.0      # outputs = the first level's four features
    m["weights"] = W
    m["biases"] = [np.full(128, 0.0, np.float32)] * 4 + [np.zeros(4, np.float32)]
    x = np.array([[0.0, 0.0, 0.0, 0.5]], np.float32)
    with nb.NatField.from_params(m) as f:
        out = f.forward(x)
    # hidden layers are identity with ReLU: the negative feature is cut to 0
    expect = np.maximum(_bf16_torch(_half_torch(vals)), 0.0)
    assert np.array_equal(out[0].astype(np.float64), expect), (out[0], expect)
    assert expect[0] != np.maximum(_bf16_torch(vals), 0.0)[0] and expect[1] == 0.0


def test_device_tensors_and_empty_input(nb):
    torch = pytest.importorskip("torch")
    m = S.nat_params(seed=5)
    x = S.nat_queries(3000, 6, 21)
    with nb.NatField.from_params(m) as f:
        xt = torch.from_numpy(x).cuda()
        out = f.forward(xt)
        torch.cuda.synchronize()
        assert out.is_cuda
        host = f.forward(x)
        assert np.array_equal(out.cpu().numpy(), host)  # one kernel, same bits
        empty = f.forward(np.zeros((0, 6), np.float32))
        assert empty.shape == (0, 8)
    _check(host, x, m)


def test_device_parameters(nb):
    """Parameters passed as CUDA tensors give the same field as host arrays."""
    torch = pytest.importorskip("torch")
    m = S.nat_params(seed=12)
    x = S.nat_queries(500, 6, 22)
    cat = lambda xs: np.concatenate([np.asarray(a, np.float32).ravel() for a in xs])
    with nb.NatField.from_params(m) as f:
        host = f.forward(x)
    dev = [torch.from_numpy(cat(m[k])).cuda() for k in ("tables", "weights", "biases")]
    with nb.NatField(m["n_cond"], m["n_out"], m["table_log2"], *dev) as f:
        out = f.forward(x)
    assert np.array_equal(out, host)


def test_full_size_sampled(nb):
    """2^22 queries (the bench's size) in one call: sampled rows against the oracle, and the
    outputs of a repeated call identical (fixed reduction order)."""
    m = S.nat_params(seed=6)
    n = 1 << 22
    x = S.nat_queries(n, 6, 31)
    with nb.NatField.from_params(m) as f:
        out = f.forward(x)
        again = f.forward(x)
    assert np.array_equal(out, again)
    rows = np.random.default_rng(3).choice(n, 4096, replace=False)
    rows = np.concatenate([rows, [0, n - 1]])
    _check(out[rows], x[rows], m)


def test_host_buffers_pipelined_match_device(nb):
    """Host inputs or outputs beyond 2^20 queries run in overlapped chunks; every query is
    independent, so the results equal one call on device buffers bit for bit (2^21 + 777
    queries: three chunks, the last ragged)."""
    torch = pytest.importorskip("torch")
    m = S.nat_params(seed=8)
    n = (1 << 21) + 777
    x = S.nat_queries(n, 6, 33)
    with nb.NatField.from_params(m) as f:
        xt = torch.from_numpy(x).cuda()
        ref = f.forward(xt)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        host = f.forward(x)                                   # host in, host out
        assert np.array_equal(host, ref)
        xp = torch.from_numpy(x).pin_memory()
        op = torch.empty((n, 8), dtype=torch.float32).pin_memory()
        st = nb.lib().nat_field_forward(f.handle, ctypes.c_void_p(xp.data_ptr()), n,
                                        ctypes.c_void_p(op.data_ptr()), None)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert np.array_equal(op.numpy(), ref)                # pinned host in and out
        od = torch.empty((n, 8), dtype=torch.float32, device="cuda")
        st = nb.lib().nat_field_forward(f.handle, ctypes.c_void_p(xp.data_ptr()), n,
                                        ctypes.c_void_p(od.data_ptr()), None)
        assert st == nb.NAT_BEM_OK
        torch.cuda.synchronize()
        assert np.array_equal(od.cpu().numpy(), ref)          # host in, device out
        oh = np.zeros((n, 8), np.float32)
        st = nb.lib().nat_field_forward(f.handle, ctypes.c_void_p(xt.data_ptr()), n,
                                        ctypes.c_void_p(oh.ctypes.data), None)
        assert st == nb.NAT_BEM_OK
        assert np.array_equal(oh, ref)                        # device in, host out
