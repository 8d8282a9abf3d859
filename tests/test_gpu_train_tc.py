"""Tensor-core (tcgen05) training of the SR generator (GPU).

With W a multiple of 128 the trainer runs its 64- and 256-channel
convolutions (forward, data gradient, weight gradient) on the tensor cores:
each GEMM rounds its two operands to bf16 (round to nearest even) and
accumulates in FP32.  The reference is torch autograd of the same network in
FP64 on the CPU (a library routine, independent of the CUDA kernels) in which
every such GEMM rounds the same operands the same way: the forward rounds the
layer input and the weights, the data gradient the output gradient and the
weights, the weight gradient the layer input and the output gradient (the
rounding is passed straight through in the backward pass).  What remains
between the two is FP32 against FP64 accumulation and, where an FP32 value
lies within its own rounding of a bf16 rounding boundary, a bf16 rounding the
other way (about 1 element in 10^4); the bounds below cover both.  Against the
unrounded FP64 network the gradients differ by the bf16 operand noise (a few
2^-9 relative per operand, averaged over the K terms of each sum), and
against the trainer's own FP32 path by the same amount.
"""
import numpy as np
import pytest

from synthetic.weights import random_weights

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NB = 2
H = W = 128
B = 1


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _case(seed):
    rng = np.random.default_rng(seed)
    w = random_weights(seed, n_blocks=NB, gain=0.7)
    q = rng.standard_normal((B, H, W))
    t = rng.standard_normal((B, 2 * H, 2 * W)) * 0.1
    mask = (rng.uniform(size=(B, 2 * H, 2 * W)) > 0.3).astype(np.float64)
    return w, q, t, mask


def _r16(x):
    """An FP64 tensor rounded as the GPU rounds its FP32 value to bf16."""
    return x.float().bfloat16().double()


def _torch_net(w, q, t, mask, bf16_gemms):
    import torch.nn.functional as Fn

    P = {k: torch.tensor(np.asarray(v, dtype=np.float32).astype(np.float64), requires_grad=True)
         for k, v in w.items()}

    def pconv(x, wt):
        return Fn.conv2d(Fn.pad(x, (1, 1, 1, 1), mode="circular"), wt)

    class TcConv(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, wt):
            xr, wr = _r16(x), _r16(wt)
            ctx.save_for_backward(xr, wr)
            return pconv(xr, wr)

        @staticmethod
        def backward(ctx, g):
            xr, wr = ctx.saved_tensors
            with torch.enable_grad():
                xa = xr.detach().requires_grad_(True)
                wa = wr.detach().requires_grad_(True)
                dx, dw = torch.autograd.grad(pconv(xa, wa), (xa, wa), _r16(g))
            return dx, dw

    def conv(x, wk, bk, wide=True):
        y = TcConv.apply(x, P[wk]) if (wide and bf16_gemms) else pconv(x, P[wk])
        return y + P[bk][None, :, None, None]

    x = torch.tensor(np.asarray(q, dtype=np.float32).astype(np.float64))[:, None]
    x = Fn.prelu(conv(x, "in.w", "in.b", wide=False), P["in.a"])
    for k in range(NB):
        a = Fn.prelu(conv(x, f"b{k}.w1", f"b{k}.b1"), P[f"b{k}.a"])
        x = x + conv(a, f"b{k}.w2", f"b{k}.b2")
    u = Fn.prelu(Fn.pixel_shuffle(conv(x, "up.w", "up.b"), 2), P["up.a"])
    y = conv(u, "out.w", "out.b", wide=False)[:, 0]
    tt = torch.tensor(np.asarray(t, dtype=np.float32).astype(np.float64))
    loss = (torch.tensor(mask) * (y - tt) ** 2).sum() / y.numel()
    loss.backward()
    return loss.item(), {k: v.grad.numpy() for k, v in P.items()}, y.detach().numpy()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def _groups(g, n_blocks):
    from paper_2403_07936_gb300 import sr
    out, off = {}, 0
    for name, shape in sr.layer_order(64, n_blocks):
        k = int(np.prod(shape))
        out[name] = g[off:off + k].reshape(shape)
        off += k
    return out


def _grads(mg, blob, q, t, mask, tensor_cores):
    tr = mg.Trainer(H, W, B, blob)
    tr.tensor_cores = tensor_cores
    n = (len(blob) - 64) // 4
    g = torch.empty(n, device=DEV)
    y = torch.empty((B, 2 * H, 2 * W), device=DEV)
    loss = tr.gradients(_dev(q), _dev(t), g, mask=_dev(mask))
    tr.forward(_dev(q), y)
    torch.cuda.synchronize()
    return loss, _groups(g.cpu().numpy().astype(np.float64), NB), y.double().cpu().numpy()


def test_tensor_cores_are_the_default_for_rows_of_whole_tiles(mg):
    from paper_2403_07936_gb300 import sr
    blob = sr.pack_weights(random_weights(1, n_blocks=NB), n_blocks=NB)
    assert mg.Trainer(H, W, B, blob).tensor_cores
    small = mg.Trainer(16, 16, 8, blob)
    assert not small.tensor_cores
    with pytest.raises(mg.MGError):
        small.tensor_cores = True
    tr = mg.Trainer(H, W, B, blob)
    tr.tensor_cores = False
    assert not tr.tensor_cores


def test_tensor_core_forward_and_gradients_match_bf16_operand_autograd(mg):
    from paper_2403_07936_gb300 import sr
    w, q, t, mask = _case(5)
    blob = sr.pack_weights(w, n_blocks=NB)
    loss, g, y = _grads(mg, blob, q, t, mask, True)
    ref_loss, ref_g, ref_y = _torch_net(w, q, t, mask, bf16_gemms=True)
    # forward: element by element
    assert np.abs(y[0] - ref_y[0]).max() <= 2e-3 * np.abs(ref_y).max()
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    for name, ref in ref_g.items():
        got = g[name]
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err <= 5e-3, (name, err)
        # element by element, against the group's largest entry
        assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max(), name


def test_tensor_core_gradients_are_the_fp32_gradients_up_to_bf16_noise(mg):
    from paper_2403_07936_gb300 import sr
    w, q, t, mask = _case(6)
    blob = sr.pack_weights(w, n_blocks=NB)
    _, g_tc, y_tc = _grads(mg, blob, q, t, mask, True)
    _, g_32, y_32 = _grads(mg, blob, q, t, mask, False)
    _, ref_g, _ = _torch_net(w, q, t, mask, bf16_gemms=False)
    assert np.abs(y_tc - y_32).max() <= 3e-2 * np.abs(y_32).max()
    for name, ref in ref_g.items():
        e32 = np.linalg.norm(g_32[name] - ref) / max(np.linalg.norm(ref), 1e-30)
        etc = np.linalg.norm(g_tc[name] - ref) / max(np.linalg.norm(ref), 1e-30)
        assert e32 <= 2e-4, (name, e32)
        assert etc <= 5e-2, (name, etc)


def test_tensor_core_adam_steps_lower_the_loss_on_a_teacher(mg):
    from oracle import generator as og
    from paper_2403_07936_gb300 import sr
    rng = np.random.default_rng(7)
    teacher = random_weights(40, n_blocks=NB, gain=0.7)
    q = rng.standard_normal((B, H, W))
    w32 = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in teacher.items()}
    t = og.generator_forward(np.asarray(q[0], dtype=np.float32).astype(np.float64), w32, n_blocks=NB)[None]
    tr = mg.Trainer(H, W, B, sr.pack_weights(random_weights(41, n_blocks=NB, gain=0.7), n_blocks=NB), lr=1e-3)
    assert tr.tensor_cores
    qd, td = _dev(q), _dev(t)
    losses = [tr.step(qd, td) for _ in range(60)]
    assert np.isfinite(losses).all() and losses[-1] < 0.5 * losses[0], losses[::10]
