"""The bounds-checked build (libseb_debug.so, compiled with -DSEB_DEBUG): every index of the
staged tile, of the row runs and of the output stores is checked in the kernel, and a failed
check raises a bit of the device error word instead of touching memory.  A child process runs
the map paths on it (rebuild and rolling shifts with the TMA staging, shifts whose column bands
take the column layouts, a ragged map with plain loads, the compensated sums, the tiled BF16
storage, and a footprint whose packed missing-point moments are flushed); seb_map_check must find
the error word
clear, and the outputs must equal the release build's bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2503_02412_gb300 as seb
from synthetic import fractal_world, fractal_steps_nan, shift_sequence
C2 = dict(n_yaw=72, res=0.05, length=0.9, width=0.6)
res = {}
world = torch.from_numpy(fractal_world(3, 420)).cuda()
n = 160
win = lambda o: world[o[1]:o[1] + n, o[0]:o[0] + n].contiguous()
m = seb.SebMap(seb.SebParams(nx=n, ny=n, **C2))
o = [130, 130]
m.update(win(o), tuple(o))
moves = list(shift_sequence(5, 8, 9))
for dx, dy in moves[:4]:
    o = [o[0] + dx, o[1] + dy]
    m.shift(win(o), tuple(o))
origins = []
for dx, dy in moves[4:]:
    o = [o[0] + dx, o[1] + dy]
    origins.append(tuple(o))
m.shift_batch([win(q) for q in origins], origins)
out, fl = m.outputs()
m.check()
res["rolling"] = out.cpu().numpy()
res["rolling_flags"] = fl.cpu().numpy()
e = torch.from_numpy(fractal_steps_nan(4, 37, 53, nan_frac=0.04)).cuda()
m = seb.SebMap(seb.SebParams(nx=37, ny=53, **C2))
m.update(e)
res["ragged"] = m.outputs()[0].cpu().numpy()
m.check()
e = torch.from_numpy(fractal_steps_nan(6, n, n)).cuda()
m = seb.SebMap(seb.SebParams(nx=n, ny=n, precision="compensated", **C2))
m.update(e)
res["compensated"] = m.outputs()[0].cpu().numpy()
m.check()
m = seb.SebMap(seb.SebParams(nx=n, ny=n, elev_dtype="bf16_tiled", **C2))
m.update(seb.encode_bf16_tiled(e), (0, 0))
res["tiled"] = m.outputs()[0].cpu().numpy()
m.check()
# moves whose column bands are 3, 4 and 5 blocks wide (column layouts, piece cutting)
m = seb.SebMap(seb.SebParams(nx=n, ny=n, **C2))
o = [130, 130]
m.update(win(o), tuple(o))
for dx, dy in [(2, 0), (10, 1), (-6, 0), (-13, 2), (17, -3)]:
    o = [o[0] + dx, o[1] + dy]
    m.shift(win(o), tuple(o))
res["bands"] = m.outputs()[0].cpu().numpy()
m.check()
# a footprint whose missing-point moments are flushed from the packed words every few runs
F = dict(n_yaw=4, res=0.05, length=1.3, width=0.9)
m = seb.SebMap(seb.SebParams(nx=96, ny=72, **F))
m.update(world[100:172, 100:196].contiguous(), (100, 100))
m.shift(world[97:169, 104:200].contiguous(), (104, 97))
res["flushed"] = m.outputs()[0].cpu().numpy()
m.check()
np.savez(sys.argv[2], **res)
print("library", seb.abi.LIB_PATH)
'''


def run_child(lib, out):
    env = dict(os.environ)
    if lib:
        env["SEB_LIBRARY"] = lib
    else:
        env.pop("SEB_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, out], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_bounds_checked_build_is_clean_and_identical(tmp_path):
    import __graft_entry__
    from paper_2503_02412_gb300 import build

    __graft_entry__.build()
    dbg = build.build(debug=True)
    a = run_child(dbg, str(tmp_path / "debug.npz"))
    b = run_child(None, str(tmp_path / "release.npz"))
    for k in b.files:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k
