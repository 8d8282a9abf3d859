"""Training kernels of the SR generator (GPU).

The trainer's forward pass is compared with the FP64 generator oracle, its
gradients with torch autograd of the same network in FP64 on the CPU (a
library reference, independent of the CUDA kernels), and a few Adam steps on
a teacher network's outputs must lower the loss.  Tolerances: forward 1e-5
relative (FP32 accumulation over K <= 2304 terms per layer, 20 layers);
gradients 2e-4 relative per parameter group in the 2-norm (FP32 sums over
2048 pixels and the chained backward pass).
"""
import numpy as np
import pytest

from oracle import generator as og
from synthetic.weights import random_weights

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NB = 2
H = W = 16
B = 8


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


def _torch_loss(w, q, t, mask):
    import torch.nn.functional as Fn
    P = {k: torch.tensor(np.asarray(v, dtype=np.float32).astype(np.float64), requires_grad=True)
         for k, v in w.items()}

    def conv(x, wk, bk):
        return Fn.conv2d(Fn.pad(x, (1, 1, 1, 1), mode="circular"), P[wk], P[bk])

    x = torch.tensor(np.asarray(q, dtype=np.float32).astype(np.float64))[:, None]
    x = Fn.prelu(conv(x, "in.w", "in.b"), P["in.a"])
    for k in range(NB):
        a = Fn.prelu(conv(x, f"b{k}.w1", f"b{k}.b1"), P[f"b{k}.a"])
        x = x + conv(a, f"b{k}.w2", f"b{k}.b2")
    u = Fn.prelu(Fn.pixel_shuffle(conv(x, "up.w", "up.b"), 2), P["up.a"])
    y = conv(u, "out.w", "out.b")[:, 0]
    tt = torch.tensor(np.asarray(t, dtype=np.float32).astype(np.float64))
    m = torch.tensor(mask)
    loss = (m * (y - tt) ** 2).sum() / y.numel()
    loss.backward()
    return loss.item(), {k: v.grad.numpy() for k, v in P.items()}, y.detach().numpy()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def test_forward_matches_generator_oracle(mg):
    from paper_2403_07936_gb300 import sr
    w, q, _, _ = _case(1)
    tr = mg.Trainer(H, W, B, sr.pack_weights(w, n_blocks=NB))
    y = torch.empty((B, 2 * H, 2 * W), device=DEV)
    tr.forward(_dev(q), y)
    torch.cuda.synchronize()
    got = y.double().cpu().numpy()
    w32 = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in w.items()}
    for b in range(B):
        ref = og.generator_forward(np.asarray(q[b], dtype=np.float32).astype(np.float64), w32, n_blocks=NB)
        assert np.abs(got[b] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_gradients_match_torch_autograd(mg):
    from paper_2403_07936_gb300 import sr
    w, q, t, mask = _case(2)
    tr = mg.Trainer(H, W, B, sr.pack_weights(w, n_blocks=NB))
    blob = sr.pack_weights(w, n_blocks=NB)
    n = (len(blob) - 64) // 4
    g = torch.empty(n, device=DEV)
    loss = tr.gradients(_dev(q), _dev(t), g, mask=_dev(mask))
    torch.cuda.synchronize()
    ref_loss, ref_g, _ = _torch_loss(w, q, t, mask)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    gh = g.cpu().numpy().astype(np.float64)
    off = 0
    for name, shape in sr.layer_order(64, NB):
        k = int(np.prod(shape))
        got, ref = gh[off:off + k].reshape(shape), ref_g[name]
        off += k
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err <= 2e-4, (name, err)


def test_adam_steps_lower_the_loss_on_a_teacher(mg):
    from paper_2403_07936_gb300 import sr
    rng = np.random.default_rng(3)
    teacher = random_weights(30, n_blocks=NB, gain=0.7)
    q = rng.standard_normal((B, H, W))
    w32 = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in teacher.items()}
    t = np.stack([og.generator_forward(np.asarray(q[b], dtype=np.float32).astype(np.float64), w32, n_blocks=NB)
                  for b in range(B)])
    student = random_weights(31, n_blocks=NB, gain=0.7)
    blob0 = sr.pack_weights(student, n_blocks=NB)
    tr = mg.Trainer(H, W, B, blob0, lr=1e-3)
    assert tr.weights() == blob0  # no step yet: the blob round-trips exactly
    qd, td = _dev(q), _dev(t)
    losses = [tr.step(qd, td) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], losses[::10]
    w1 = sr.unpack_weights(tr.weights())
    assert set(w1) == set(student) and any(np.any(w1[k] != np.float32(student[k])) for k in w1)


def test_trainer_rejects_bad_shapes(mg):
    from paper_2403_07936_gb300 import sr
    blob = sr.pack_weights(random_weights(1, n_blocks=NB), n_blocks=NB)
    for h, w_, b in [(12, 16, 8), (16, 16, 1), (4, 4, 128)]:
        with pytest.raises(mg.MGError):
            mg.Trainer(h, w_, b, blob)
    with pytest.raises(mg.MGError):
        mg.Trainer(H, W, B, blob[:-4])
