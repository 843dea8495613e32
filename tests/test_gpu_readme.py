"""The quick-start usage shown in README.md, run as written on a small map: rebuild, rolling
shift, outputs, a map channel as an SE(2) grid, its SDF, the trilinear lookup with gradients and
the exact continuous query with its autograd backward."""
import numpy as np
import pytest

from synthetic import fractal_world, random_poses

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_quick_start_usage():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2503_02412_gb300 as seb
    from paper_2503_02412_gb300.query import QueryPoses

    n, res = 100, 0.05
    world = torch.from_numpy(fractal_world(3, 300, res)).cuda()
    oi, oj = 40, 60
    elev = world[oj:oj + n, oi:oi + n].contiguous()
    next_elev = world[oj - 3:oj - 3 + n, oi + 10:oi + 10 + n].contiguous()

    p = seb.SebParams(nx=n, ny=n, n_yaw=72, res=res, length=0.9, width=0.6)
    m = seb.SebMap(p)
    m.update(elev, origin=(oi, oj))
    m.shift(next_elev, origin=(oi + 10, oj - 3))
    origins = [(oi + 10 + 2 * k, oj - 3 - k) for k in range(1, 4)]
    windows = [world[q[1]:q[1] + n, q[0]:q[0] + n].contiguous() for q in origins]
    m.shift_batch(windows, origins)
    m.shift(world[oj - 3:oj - 3 + n, oi + 10:oi + 10 + n].contiguous(), origin=(oi + 10, oj - 3))
    out, flags = m.outputs()
    assert tuple(out.shape) == (5, 72, n, n) and tuple(flags.shape) == (72, n, n)
    m.check()

    risk = seb.SE2Grid.from_map(m, 4)
    sdf = seb.risk_sdf(risk, risk_obstacle=1.0, clamp=2.0)
    poses = torch.from_numpy(random_poses(5, 1000, n, n, res, 12, origin=(oi + 10, oj - 3))).cuda()
    val, grad, fl = seb.se2_lookup(sdf, poses, with_grad=True)
    assert val.shape == (1000,) and grad.shape == (1000, 3) and bool((fl == 0).any())
    assert bool(torch.isfinite(val[fl == 0]).all())

    q = poses.clone().requires_grad_()
    out_q, fl_q = QueryPoses.apply(q, next_elev, p, (oi + 10, oj - 3))
    out_q[:, 4].sum().backward()
    assert out_q.shape == (1000, 5) and q.grad is not None and bool(torch.isfinite(q.grad).all())
    ok = (fl_q == 0).cpu().numpy()
    assert ok.mean() > 0.5 and np.isfinite(out_q.detach().cpu().numpy()[ok]).all()
