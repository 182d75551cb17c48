"""Tensor-core convolution kernels vs the FP64 oracle (inputs pre-rounded to
BF16 so both sides see the same values; FP32 outputs within 1e-4 of the
maximum, BF16 outputs within BF16 rounding), the element-wise kernels vs
numpy, and the learned few-view correction end to end on a small scan."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2104_13248_gb300 import _lib, inputs, learned
from paper_2104_13248_gb300.unet import UNet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def P(t):
    return ctypes.c_void_p(t.data_ptr())


def S():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


SHAPES = [(1, 8, 8, 16, 16, 16), (2, 6, 9, 13, 32, 64), (1, 12, 10, 9, 48, 16), (1, 4, 4, 20, 96, 32),
          (1, 16, 16, 16, 64, 64)]
# layers the tcgen05 kernels take: width a multiple of 128 with Cout 16 / 32, or a
# multiple of 64 (not of 128) with Cout 16 / 32 / 64 (tiles of 64 voxels, M = 64
# MMAs); depth a multiple of 4
TC_SHAPES = [(1, 4, 2, 128, 16, 16), (1, 4, 3, 256, 48, 16), (2, 4, 3, 128, 32, 32), (1, 8, 1, 128, 96, 32),
             (1, 8, 5, 256, 32, 16), (2, 12, 3, 128, 16, 32),
             (1, 4, 3, 64, 32, 64), (2, 4, 2, 64, 64, 64), (1, 8, 3, 192, 64, 32), (1, 4, 5, 64, 16, 16)]


@pytest.mark.parametrize("path", [1, 2, 0], ids=["tcgen05_persistent", "tcgen05_tile", "mma_sync"])
@pytest.mark.parametrize("shape", TC_SHAPES, ids=lambda s: "n%d_%dx%dx%d_ci%d_co%d" % s)
def test_conv_tensor_core_paths(shape, path):
    """The tcgen05 / TMEM kernel (and, forced, the mma.sync kernel) on the
    same layers: forward FP32 and BF16 (ReLU, channel slice of a wider
    tensor) and the input gradient, all against the FP64 oracle."""
    lib = _lib.load()
    _lib.check(lib.cnn_set_tensor_path(path))
    try:
        test_conv_forward_dgrad_wgrad(shape)
        _lib.check(lib.cnn_device_status(S()))
    finally:
        _lib.check(lib.cnn_set_tensor_path(1))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "n%d_%dx%dx%d_ci%d_co%d" % s)
def test_conv_forward_dgrad_wgrad(shape):
    n, d, h, w, cin, cout = shape
    rng = np.random.default_rng(sum(shape))
    x = bf16_round(rng.normal(size=(n, d, h, w, cin)))
    wt = bf16_round(rng.normal(size=(cout, 27, cin)) * 0.1)
    b = rng.normal(size=cout).astype(np.float32)
    dy = bf16_round(rng.normal(size=(n, d, h, w, cout)))
    xd = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    wd = torch.from_numpy(wt.astype(np.float32)).cuda().to(torch.bfloat16)
    bd = torch.from_numpy(b).cuda()
    dyd = torch.from_numpy(dy.astype(np.float32)).cuda().to(torch.bfloat16)
    lib = _lib.load()
    # forward, FP32 output, bias, no ReLU
    y32 = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
    _lib.check(lib.cnn_conv3d_forward(P(xd), cin, 0, P(wd), P(bd), P(y32), cout, 0, 1, n, d, h, w, cin, cout, 0, S()))
    ref = oracle.conv3d(x, wt, b)
    assert rel(y32.cpu().numpy(), ref) <= 1e-4
    # forward, BF16 output with ReLU, written into a channel slice of a wider tensor
    ybig = torch.zeros((n, d, h, w, cout + 16), dtype=torch.bfloat16, device="cuda")
    _lib.check(lib.cnn_conv3d_forward(P(xd), cin, 0, P(wd), P(bd), P(ybig), cout + 16, 16, 0, n, d, h, w, cin,
                                      cout, 1, S()))
    yb = ybig.float().cpu().numpy()
    assert rel(yb[..., 16:], np.maximum(ref, 0)) <= 8e-3
    assert np.all(yb[..., :16] == 0)
    # input gradient (BF16 out)
    dx = torch.empty((n, d, h, w, cin), dtype=torch.bfloat16, device="cuda")
    scratch = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device="cuda")
    _lib.check(lib.cnn_conv3d_dgrad(P(dyd), cout, 0, P(wd), P(scratch), P(dx), cin, 0, n, d, h, w, cin, cout, S()))
    dref = oracle.conv3d_dgrad(dy, wt)
    assert rel(dx.float().cpu().numpy(), dref) <= 8e-3
    # the same input gradient at FP32 through the forward kernel and the flipped weights
    if cin in (16, 32, 64):
        dx32 = torch.empty((n, d, h, w, cin), dtype=torch.float32, device="cuda")
        _lib.check(lib.cnn_conv3d_forward(P(dyd), cout, 0, P(scratch), None, P(dx32), cin, 0, 1, n, d, h, w, cout,
                                          cin, 0, S()))
        assert rel(dx32.cpu().numpy(), dref) <= 1e-4
    # weight and bias gradients (FP32, accumulated onto the initial values)
    dw = torch.full((cout, 27, cin), 0.5, dtype=torch.float32, device="cuda")
    db = torch.full((cout,), -0.25, dtype=torch.float32, device="cuda")
    _lib.check(lib.cnn_conv3d_wgrad(P(xd), cin, 0, P(dyd), cout, 0, P(dw), P(db), n, d, h, w, cin, cout, S()))
    wref, bref = oracle.conv3d_wgrad(x, dy)
    assert rel(dw.cpu().numpy() - 0.5, wref) <= 1e-4
    assert rel(db.cpu().numpy() + 0.25, bref) <= 1e-4


def test_pool_upsample_relu():
    rng = np.random.default_rng(5)
    n, d, h, w, c = 2, 6, 4, 8, 16
    x = bf16_round(rng.normal(size=(n, d, h, w, c + 16)))
    xd = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    lib = _lib.load()
    y = torch.empty((n, d // 2, h // 2, w // 2, c), dtype=torch.bfloat16, device="cuda")
    _lib.check(lib.cnn_maxpool2_forward(P(xd), c + 16, 16, P(y), n, d, h, w, c, S()))
    xs = x[..., 16:].reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c)
    ref = xs.max(axis=(2, 4, 6))
    assert np.array_equal(y.float().cpu().numpy(), ref)
    # backward adds dy at the first arg-max of each window
    dy = bf16_round(rng.normal(size=ref.shape))
    dyd = torch.from_numpy(dy.astype(np.float32)).cuda().to(torch.bfloat16)
    dx = torch.zeros((n, d, h, w, c + 16), dtype=torch.bfloat16, device="cuda")
    _lib.check(lib.cnn_maxpool2_backward(P(xd), c + 16, 16, P(dyd), P(dx), c + 16, 16, n, d, h, w, c, S()))
    got = dx.float().cpu().numpy()[..., 16:].reshape(xs.shape)
    flat = xs.transpose(0, 1, 3, 5, 7, 2, 4, 6).reshape(n, d // 2, h // 2, w // 2, c, 8)
    arg = flat.argmax(axis=-1)
    exp = np.zeros_like(flat)
    np.put_along_axis(exp, arg[..., None], dy[..., None], axis=-1)
    exp = exp.reshape(n, d // 2, h // 2, w // 2, c, 2, 2, 2).transpose(0, 1, 5, 2, 6, 3, 7, 4)
    assert np.array_equal(got, exp)
    # upsample forward into a channel slice, backward sums the 8 children
    up = torch.zeros((n, d * 2, h * 2, w * 2, c + 8), dtype=torch.bfloat16, device="cuda")
    src = xd[..., 16:].contiguous()
    _lib.check(lib.cnn_upsample2_forward(P(src), P(up), c + 8, 8, n, d, h, w, c, S()))
    u = up.float().cpu().numpy()[..., 8:]
    assert np.array_equal(u, x[..., 16:].repeat(2, 1).repeat(2, 2).repeat(2, 3))
    gsum = torch.empty((n, d, h, w, c), dtype=torch.bfloat16, device="cuda")
    _lib.check(lib.cnn_upsample2_backward(P(up), c + 8, 8, P(gsum), n, d, h, w, c, S()))
    assert rel(gsum.float().cpu().numpy(), 8 * x[..., 16:]) <= 4e-3
    # ReLU backward masks where y <= 0
    g = torch.ones((n, d, h, w, c), dtype=torch.bfloat16, device="cuda")
    _lib.check(lib.cnn_relu_backward(P(g), c, 0, P(xd), c + 16, 16, n * d * h * w, c, S()))
    assert np.array_equal(g.float().cpu().numpy(), (x[..., 16:] > 0).astype(np.float32))


@pytest.mark.parametrize("shape", [(1, 8, 12, 16, 16), (2, 5, 7, 20, 16), (1, 4, 4, 8, 32), (1, 6, 9, 132, 8)],
                         ids=lambda s: "n%d_%dx%dx%d_co%d" % s)
def test_stem_forward_wgrad(shape):
    """The one-channel input layer (tcgen05 at widths that are multiples of
    8, mma.sync otherwise) against the FP64 oracle's
    convolution with Cin = 1, the input pre-rounded to BF16 as the kernel
    rounds it: forward FP32-accurate before the BF16 store, weight and bias
    gradients within 1e-4."""
    n, d, h, w, cout = shape
    rng = np.random.default_rng(sum(shape) + 7)
    x = rng.normal(size=(n, d, h, w)).astype(np.float32)
    xb = bf16_round(x)
    wt = bf16_round(rng.normal(size=(cout, 27, 1)) * 0.2)
    b = rng.normal(size=cout).astype(np.float32)
    dy = bf16_round(rng.normal(size=(n, d, h, w, cout)))
    lib = _lib.load()
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(wt.astype(np.float32)).cuda().to(torch.bfloat16)
    bd = torch.from_numpy(b).cuda()
    ref = oracle.conv3d(xb[..., None], wt, b)
    for relu in (0, 1):
        y = torch.zeros((n, d, h, w, cout + 8), dtype=torch.bfloat16, device="cuda")
        _lib.check(lib.cnn_stem_forward(P(xd), P(wd), P(bd), P(y), cout + 8, 8, n, d, h, w, cout, relu, S()))
        yb = y.float().cpu().numpy()
        exp = np.maximum(ref, 0) if relu else ref
        assert rel(yb[..., 8:], exp) <= 8e-3                      # BF16 output rounding
        assert np.all(yb[..., :8] == 0)
    dyd = torch.from_numpy(dy.astype(np.float32)).cuda().to(torch.bfloat16)
    dw = torch.full((cout, 27), 0.5, dtype=torch.float32, device="cuda")
    db = torch.full((cout,), -0.25, dtype=torch.float32, device="cuda")
    _lib.check(lib.cnn_stem_wgrad(P(xd), P(dyd), cout, 0, P(dw), P(db), n, d, h, w, cout, S()))
    wref, bref = oracle.conv3d_wgrad(xb[..., None], dy)
    assert rel(dw.cpu().numpy() - 0.5, wref[..., 0]) <= 1e-4
    assert rel(db.cpu().numpy() + 0.25, bref) <= 1e-4
    _lib.check(lib.cnn_device_status(S()))


def test_stem_rejects_bad_layouts():
    lib = _lib.load()
    x = torch.zeros(64, device="cuda")
    w = torch.zeros(16 * 27, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(64 * 16, dtype=torch.bfloat16, device="cuda")
    assert lib.cnn_stem_forward(P(x), P(w), None, P(y), 16, 0, 1, 4, 4, 3, 16, 1, S()) == _lib.BP_ERR_INVALID_ARG
    assert lib.cnn_stem_forward(P(x), P(w), None, P(y), 16, 0, 1, 4, 4, 4, 12, 1, S()) == _lib.BP_ERR_INVALID_ARG
    assert lib.cnn_stem_wgrad(P(x), P(y), 16, 8, P(x), None, 1, 4, 4, 4, 16, S()) == _lib.BP_ERR_INVALID_ARG


@pytest.mark.parametrize("dims", [(1, 4, 130, 16), (2, 5, 12, 8), (1, 6, 128, 24), (1, 2, 256, 40)],
                         ids=["ragged_h", "odd_d_batch2", "tile_h", "two_y_tiles"])
def test_stem_tensor_core_against_oracle_and_mma_sync(dims):
    """The tcgen05 input layer (x taps in K, banded weights): a channel slice
    of a wider output, ragged y tiles, an odd depth, a batch of two and a
    single x tile whose halo lies outside on both sides. Against the FP64
    oracle within BF16 output rounding, against the mma.sync kernel on the
    same inputs within one BF16 step (the two sum the same products in
    different orders), and with the pooling (where d and h are even) bit for
    bit the separate pooling."""
    n, d, h, w = dims
    lib = _lib.load()
    rng = np.random.default_rng(sum(dims) + 3)
    x = rng.normal(size=(n, d, h, w)).astype(np.float32)
    wt = bf16_round(rng.normal(size=(16, 27, 1)) * 0.2)
    b = rng.normal(size=16).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    wd = torch.from_numpy(wt.astype(np.float32)).cuda().to(torch.bfloat16)
    bd = torch.from_numpy(b).cuda()
    ref = np.maximum(oracle.conv3d(bf16_round(x)[..., None], wt, b), 0)
    outs = []
    for path in (1, 0):
        _lib.check(lib.cnn_set_tensor_path(path))
        try:
            y = torch.zeros((n, d, h, w, 24), dtype=torch.bfloat16, device="cuda")
            _lib.check(lib.cnn_stem_forward(P(xd), P(wd), P(bd), P(y), 24, 8, n, d, h, w, 16, 1, S()))
            _lib.check(lib.cnn_device_status(S()))
        finally:
            _lib.check(lib.cnn_set_tensor_path(1))
        yb = y.float().cpu().numpy()
        assert np.all(yb[..., :8] == 0)
        assert rel(yb[..., 8:], ref) <= 8e-3
        outs.append(yb[..., 8:])
    tc, ms = outs
    step = np.maximum(np.abs(tc), np.abs(ms)) * 2.0 ** -7 + 1e-5   # sums near zero may differ in sign before ReLU
    assert np.all(np.abs(tc - ms) <= step)
    if d % 2 == 0 and h % 2 == 0:
        y1 = torch.zeros((n, d, h, w, 24), dtype=torch.bfloat16, device="cuda")
        y2 = torch.zeros_like(y1)
        p1 = torch.empty((n, d // 2, h // 2, w // 2, 16), dtype=torch.bfloat16, device="cuda")
        p2 = torch.empty_like(p1)
        _lib.check(lib.cnn_stem_forward(P(xd), P(wd), P(bd), P(y1), 24, 8, n, d, h, w, 16, 1, S()))
        ys = y1[..., 8:].contiguous()
        _lib.check(lib.cnn_maxpool2_forward(P(ys), 16, 0, P(p1), n, d, h, w, 16, S()))
        _lib.check(lib.cnn_stem_pool_forward(P(xd), P(wd), P(bd), P(y2), 24, 8, P(p2), n, d, h, w, 16, 1, S()))
        _lib.check(lib.cnn_device_status(S()))
        assert torch.equal(y1, y2)
        assert torch.equal(p1, p2)


def test_head1_forward_backward():
    """The 1x1x1 head and its gradients against numpy in FP64 (BF16 inputs)."""
    rng = np.random.default_rng(12)
    nvox, cs, cin = 1000, 24, 16
    x = bf16_round(rng.normal(size=(nvox, cs)))
    w = rng.normal(size=cin).astype(np.float32)
    b = np.float32(0.3)
    res = rng.normal(size=nvox).astype(np.float32)
    g = rng.normal(size=nvox).astype(np.float32)
    xd = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    wd, bd = torch.from_numpy(w).cuda(), torch.tensor([b], device="cuda")
    rd, gd = torch.from_numpy(res).cuda(), torch.from_numpy(g).cuda()
    out = torch.empty(nvox, device="cuda")
    lib = _lib.load()
    _lib.check(lib.cnn_head1_forward(P(xd), cs, P(wd), P(bd), P(rd), P(out), nvox, cin, S()))
    ref = res + b + x[:, :cin] @ w.astype(np.float64)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    dx = torch.zeros((nvox, 16), dtype=torch.bfloat16, device="cuda")
    dw = torch.full((cin,), 0.5, device="cuda")
    db = torch.full((1,), -0.25, device="cuda")
    _lib.check(lib.cnn_head1_backward(P(xd), cs, P(wd), P(gd), P(dx), 16, P(dw), P(db), nvox, cin, S()))
    assert rel(dx.float().cpu().numpy(), g[:, None].astype(np.float64) * w[None, :]) <= 4e-3
    assert rel(dw.cpu().numpy() - 0.5, g.astype(np.float64) @ x[:, :cin]) <= 1e-5
    assert abs(float(db.item()) + 0.25 - g.astype(np.float64).sum()) <= 1e-4 * np.abs(g).sum()


def test_upsample_add():
    """Nearest 2x upsampling plus a skip tensor: the FP32 sum of two BF16
    values rounded once to BF16, bit for bit."""
    rng = np.random.default_rng(11)
    n, d, h, w, c = 2, 3, 4, 5, 16
    x = bf16_round(rng.normal(size=(n, d, h, w, c)))
    sk = bf16_round(rng.normal(size=(n, 2 * d, 2 * h, 2 * w, c + 8)))
    xd = torch.from_numpy(x.astype(np.float32)).cuda().to(torch.bfloat16)
    sd = torch.from_numpy(sk.astype(np.float32)).cuda().to(torch.bfloat16)
    y = torch.zeros((n, 2 * d, 2 * h, 2 * w, c + 16), dtype=torch.bfloat16, device="cuda")
    lib = _lib.load()
    _lib.check(lib.cnn_upsample2_add_forward(P(xd), P(sd), c + 8, 8, P(y), c + 16, 16, n, d, h, w, c, S()))
    up = x.repeat(2, 1).repeat(2, 2).repeat(2, 3)
    exp = torch.from_numpy((up.astype(np.float32) + sk[..., 8:].astype(np.float32))).to(torch.bfloat16).float()
    got = y.float().cpu()
    assert torch.equal(got[..., 16:], exp)
    assert torch.all(got[..., :16] == 0)


def _torch_reference(net, x, flat):
    """The same network in plain PyTorch FP32 on the CPU, parameters taken
    from the flat vector ``flat`` (laid out like net.params)."""
    import torch.nn.functional as F
    from paper_2104_13248_gb300.unet import LINEAR

    def conv(name, t):
        w0, b0, cin, cout = net.off[name]
        wt = flat[w0:b0].reshape(cout, 3, 3, 3, cin).permute(0, 4, 1, 2, 3)
        y = F.conv3d(t, wt, flat[b0:b0 + cout], padding=1)
        return y if name in LINEAR else F.relu(y)

    def up(t):
        return F.interpolate(t, scale_factor=2)

    t = x[None, None]
    e1 = conv("e1a", t.to(torch.bfloat16).float())   # the input layer reads BF16-rounded values
    if net.has_e1b:
        e1 = conv("e1b", e1)
    e2 = conv("e2b", conv("e2a", F.max_pool3d(e1, 2)))
    e3 = conv("e3b", conv("e3a", F.max_pool3d(e2, 2)))
    d2 = conv("d2", up(conv("u3", e3)) + e2)
    d1 = up(conv("u2", d2)) + e1
    if net.has_d1:
        d1 = conv("d1", d1)
    h0 = net.head_off
    hw = flat[h0:h0 + 16].reshape(1, 16, 1, 1, 1)
    return (F.conv3d(d1, hw, flat[h0 + 16:h0 + 17]) + t)[0, 0]


@pytest.mark.parametrize("full_res", [False, True], ids=["default", "with_e1b_d1"])
def test_unet_forward_backward_against_plain_pytorch(full_res):
    """Forward output and every layer's weight gradient vs autograd on a plain
    FP32 PyTorch copy of the network (weights rounded to BF16 like the
    kernels read them), for the default network and for the one with the
    two extra full-resolution convolutions. The kernels keep activations and
    their gradients in BF16, so the comparison allows BF16-level
    differences: outputs within 2e-2 of the maximum, gradients with cosine
    similarity above 0.99."""
    net = UNet(seed=3, e1b=full_res, d1=full_res)
    with torch.no_grad():
        net.params[net.head_off:net.head_off + 16] = torch.randn(16, device="cuda") * 0.3
    x = torch.from_numpy(inputs.uniform_array(8, (16, 16, 24), 0, 1).astype(np.float32))
    tgt = torch.from_numpy(inputs.uniform_array(9, (16, 16, 24), 0, 1).astype(np.float32))
    out = net.forward(x.cuda(), train=True).cpu()
    flat = net.params.cpu().clone()
    flat[:net.n_conv] = net.params16[:net.n_conv].float().cpu()
    for name, (_, b0, _, cout) in net.off.items():   # biases stay FP32 in the kernels
        flat[b0:b0 + cout] = net.params[b0:b0 + cout].cpu()
    flat.requires_grad_(True)
    ref = _torch_reference(net, x, flat)
    assert (out - ref).abs().max().item() <= 2e-2 * ref.abs().max().item()
    g = (2 * (out - tgt) / out.numel()).contiguous()
    net.backward(g.cuda())
    loss = ((ref - tgt) ** 2).mean()
    loss.backward()
    gref = flat.grad
    for name, cin, cout in [(k, v[2], v[3]) for k, v in net.off.items()]:
        w0, b0, _, _ = net.off[name]
        a, b = net.grads[w0:b0].cpu().double(), gref[w0:b0].double()
        cos = float((a @ b) / (a.norm() * b.norm()))
        assert cos > 0.99, (name, cos)
        assert abs(a.norm() / b.norm() - 1) < 0.05, (name, float(a.norm() / b.norm()))
    h0 = net.head_off
    a, b = net.grads[h0:h0 + 17].cpu().double(), gref[h0:h0 + 17].double()
    assert float((a @ b) / (a.norm() * b.norm())) > 0.999


def test_fused_head_matches_two_calls():
    """Inference fuses d1 and the 1x1 head into the persistent tcgen05
    kernel's epilogue (width 128: that kernel takes the layer); training runs
    the two calls. The outputs agree bit for bit; with the tensor path forced
    to mma.sync the fused call reports BP_ERR_UNSUPPORTED and inference falls
    back to the two calls."""
    net = UNet(seed=4, e1b=True, d1=True)
    with torch.no_grad():
        net.params[net.head_off:net.head_off + 16] = torch.randn(16, device="cuda") * 0.3
    x = torch.from_numpy(inputs.uniform_array(21, (1, 8, 12, 128), 0, 1).astype(np.float32)).cuda()
    a = net.forward(x, train=False).clone()
    b = net.forward(x, train=True).clone()
    assert torch.equal(a, b)
    lib = _lib.load()
    _lib.check(lib.cnn_set_tensor_path(0))
    try:
        B = net._buffers((1, 8, 12, 128), False)
        r = lib.cnn_conv3d_forward_head(P(B["a1"]), 16, 0, P(net.w16("d1")), P(net.bias("d1")), P(net.head_w()),
                                        P(net.head_b()), P(x), P(B["out"]), 1, 8, 12, 128, 16, 16, 1, S())
        assert r == _lib.BP_ERR_UNSUPPORTED
        c = net.forward(x, train=False)
        assert torch.isfinite(c).all()
    finally:
        _lib.check(lib.cnn_set_tensor_path(1))
    _lib.check(lib.cnn_device_status(S()))


@pytest.mark.parametrize("dims", [(1, 8, 8, 64), (2, 6, 10, 20), (1, 18, 14, 132)], ids=["tile", "ragged", "wide"])
def test_stem_pool_matches_stem_then_pool(dims):
    """The input layer with its 2 x 2 x 2 max pooling in one pass
    (cnn_stem_pool_forward) writes bit for bit what cnn_stem_forward and
    cnn_maxpool2_forward write, on whole and ragged tiles and into a channel
    slice of a wider output."""
    n, d, h, w = dims
    lib = _lib.load()
    g = torch.Generator(device="cuda").manual_seed(sum(dims))
    x = torch.rand((n, d, h, w), generator=g, device="cuda") * 2 - 0.5
    wt = (0.3 * torch.randn((16, 27), generator=g, device="cuda")).to(torch.bfloat16)
    b = torch.randn(16, generator=g, device="cuda") * 0.1
    y1 = torch.zeros((n, d, h, w, 24), dtype=torch.bfloat16, device="cuda")
    y2 = torch.zeros_like(y1)
    p1 = torch.empty((n, d // 2, h // 2, w // 2, 16), dtype=torch.bfloat16, device="cuda")
    p2 = torch.empty_like(p1)
    _lib.check(lib.cnn_stem_forward(P(x), P(wt), P(b), P(y1), 24, 8, n, d, h, w, 16, 1, S()))
    ys = y1[..., 8:].contiguous()
    _lib.check(lib.cnn_maxpool2_forward(P(ys), 16, 0, P(p1), n, d, h, w, 16, S()))
    _lib.check(lib.cnn_stem_pool_forward(P(x), P(wt), P(b), P(y2), 24, 8, P(p2), n, d, h, w, 16, 1, S()))
    _lib.check(lib.cnn_device_status(S()))
    assert torch.equal(y1, y2)
    assert torch.equal(p1, p2)
    assert lib.cnn_stem_pool_forward(P(x), P(wt), P(b), P(y2), 24, 8, P(p2), n, d + 1, h, w, 16, 1,
                                     S()) == _lib.BP_ERR_INVALID_ARG


def test_fused_upsample_head_matches_two_calls():
    """Inference of the default network (no convolution after the last skip)
    fuses the upsampling, the skip sum and the 1x1 head in one kernel
    (cnn_upsample2_add_head1_forward); training runs the upsampling and the
    head as two calls. The outputs agree bit for bit, also on a ragged
    width and with a channel offset into a wider skip tensor."""
    net = UNet(seed=5)
    with torch.no_grad():
        net.params[net.head_off:net.head_off + 17] = torch.randn(17, device="cuda") * 0.3
    x = torch.from_numpy(inputs.uniform_array(22, (1, 8, 12, 20), 0, 1).astype(np.float32)).cuda()
    a = net.forward(x, train=False).clone()
    b = net.forward(x, train=True).clone()
    assert torch.equal(a, b)
    lib = _lib.load()
    g = torch.Generator(device="cuda").manual_seed(6)
    xc = torch.randn((2, 3, 5, 7, 16), generator=g, device="cuda").to(torch.bfloat16)
    sk = torch.randn((2, 6, 10, 14, 32), generator=g, device="cuda").to(torch.bfloat16)
    res = torch.randn((2, 6, 10, 14), generator=g, device="cuda")
    w = torch.randn(16, generator=g, device="cuda")
    bias = torch.randn(1, generator=g, device="cuda")
    a1 = torch.empty((2, 6, 10, 14, 16), dtype=torch.bfloat16, device="cuda")
    two = torch.empty((2, 6, 10, 14), device="cuda")
    one = torch.empty_like(two)
    _lib.check(lib.cnn_upsample2_add_forward(P(xc), P(sk), 32, 16, P(a1), 16, 0, 2, 3, 5, 7, 16, S()))
    _lib.check(lib.cnn_head1_forward(P(a1), 16, P(w), P(bias), P(res), P(two), a1.numel() // 16, 16, S()))
    _lib.check(lib.cnn_upsample2_add_head1_forward(P(xc), P(sk), 32, 16, P(w), P(bias), P(res), P(one),
                                                   2, 3, 5, 7, 16, S()))
    assert torch.equal(one, two)
    assert lib.cnn_upsample2_add_head1_forward(P(xc), P(sk), 32, 20, P(w), P(bias), P(res), P(one),
                                               2, 3, 5, 7, 16, S()) == _lib.BP_ERR_INVALID_ARG
    _lib.check(lib.cnn_device_status(S()))


@pytest.mark.parametrize("full_res", [False, True], ids=["default", "with_e1b_d1"])
def test_training_reduces_loss_and_checkpoint_resume(tmp_path, full_res):
    net = UNet(seed=1, e1b=full_res, d1=full_res)
    x = torch.from_numpy(inputs.uniform_array(1, (2, 16, 16, 16), 0, 1).astype(np.float32)).cuda()
    t = (x * 0.5 + 0.1).contiguous()
    losses = [net.train_step(x, t, lr=3e-3) for _ in range(60)]
    assert np.mean(losses[-5:]) < 0.3 * np.mean(losses[:5])
    # checkpoint / resume: the continued trajectory is identical
    path = tmp_path / "ck.pt"
    torch.save(net.state_dict(), path)
    cont = [net.train_step(x, t, lr=3e-3) for _ in range(3)]
    net2 = UNet(seed=99, e1b=full_res, d1=full_res)
    net2.load_state_dict(torch.load(path))
    cont2 = [net2.train_step(x, t, lr=3e-3) for _ in range(3)]
    np.testing.assert_allclose(cont, cont2, rtol=2e-3)


def test_learned_few_view_gain_small():
    """A small version of the few-view workload: 128^3 volumes, 90 -> 15 views.
    The trained network must cut the few-view RMSE (vs the full-view FDK) on
    held-out seeds well below the plain few-view FDK's."""
    g = inputs.scaled_geom(inputs.preset("c5_learned")["geom"], np=90, nu=256, nv=256, du=0.8, dv=0.8,
                           nx=64, ny=64, nz=64, sx=1.0, sy=1.0, sz=1.0)
    maker = learned.PairMaker(g, stride=6, n_ell=20, axes=(3.0, 25.0))
    rng = np.random.default_rng(0)
    xs, ts = learned.make_training_set(maker, range(2000, 2016), 32, 4, rng)
    net = UNet(seed=0)
    # the default network (no extra full-resolution convolutions) trains
    # with four times the steps of the full one, as in the full-size workload
    learned.train(net, xs, ts, steps=1600, lr=5e-4, batch=2)
    mask = learned.fov_mask(g)
    r_few, r_net = learned.evaluate(net, maker, range(9000, 9004), mask)
    print(f"few-view RMSE {r_few:.4f}, with network {r_net:.4f}")
    assert r_net < 0.85 * r_few
    # fallback: without a network the full-view path is used
    api_vol = learned.reconstruct(maker, maker.raw, None)
    assert api_vol.shape == (g["nz"], g["ny"], g["nx"])
    maker.close()
