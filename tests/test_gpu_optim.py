"""GPU Adam step and L1 loss against the oracle (float64) on the same float32
inputs."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_adam_vs_oracle():
    import torch
    from paper_2506_21633_b300.render import adam_step
    rng = np.random.default_rng(7)
    N = 1001
    p = rng.normal(size=(N, 12)).astype(np.float32)
    m = np.zeros((N, 12), np.float32)
    v = np.zeros((N, 12), np.float32)
    lr = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    tp, tm, tv = (torch.from_numpy(x.copy()).cuda() for x in (p, m, v))
    rp, rm, rv = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 8):
        g = rng.normal(size=(N, 12)).astype(np.float32)
        tg = torch.from_numpy(g).cuda()
        adam_step(tp, tg, tm, tv, lr, step, 0.9, 0.999, 1e-15)
        oracle.adam(rp, g.astype(np.float64), rm, rv, np.array(lr), 0.9, 0.999, 1e-15, step)
    torch.cuda.synchronize()
    got = tp.cpu().numpy().astype(np.float64)
    # every update moves a parameter by ~lr; compare the displacement
    disp = np.abs(rp - p.astype(np.float64)).max()
    assert np.abs(got - rp).max() <= 1e-4 * disp + 1e-6
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-5, atol=1e-6)
    assert np.allclose(tv.cpu().numpy(), rv, rtol=1e-5, atol=1e-7)


def test_l1_vs_oracle():
    import torch
    from paper_2506_21633_b300.render import l1_loss
    rng = np.random.default_rng(8)
    S = rng.normal(size=100003).astype(np.float32)
    T = rng.normal(size=100003).astype(np.float32)
    T[::7] = S[::7]  # exact ties: sign(0) = 0
    loss, g = l1_loss(torch.from_numpy(S).cuda(), torch.from_numpy(T).cuda())
    torch.cuda.synchronize()
    ref_loss, ref_g = oracle.l1([S.astype(np.float64)], [T.astype(np.float64)])
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    assert np.array_equal(np.sign(g.cpu().numpy()), np.sign(ref_g[0]))
    assert np.allclose(g.cpu().numpy(), ref_g[0], rtol=1e-6, atol=0)
