"""The bounds-checked build (nvcc -DSHT_CHECK), in place of a memory checker: every kernel index
computed from the plan tables (ring, m, coefficient index, pixel offset, scratch length) is tested
before the access, and a failed test skips the access and sets bit 1 of the plan status word.  On
small cases of every entry point the checked build must give the oracle's results and leave that
bit clear.  It runs in a child process that loads the checked library instead of the normal one."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[2])
from paper_1106_0159_gb300 import _build, sht, inputs, batch
import oracle
from oracle import geometry
lib = sys.argv[1]
_build.build = lambda *a, **k: lib
sht._LIB_PATH = lib
sht.load()

def rel(x, ref):
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))

def clean(p, what):
    st = p.device_status()
    assert st == 0, (what, st)

L, geom = 64, geometry.healpix(32)
p = sht.Plan(geom, L, L, grid=sht.GRID_HEALPIX)
a = inputs.gaussian_alm(L, L, seed=61, nmaps=2)
for mode, tol in ((sht.MODE_FP64, 1e-11), (sht.MODE_SPLIT_BF16, 1e-9)):
    p.set_mode(mode)
    s = p.alm2map(torch.from_numpy(a).cuda())
    b = p.map2alm(s).cpu().numpy()
    s = s.cpu().numpy()
    ref = oracle.alm2map_exact(geom, a[1], L, L)
    assert rel(s[1], ref) < tol, (mode, rel(s[1], ref))
    assert rel(b[1], oracle.map2alm_exact(geom, s[1], L, L)) < tol
    o = torch.empty((2, p.npix), dtype=torch.float64, device="cuda")
    p.alm2map_noalloc(torch.from_numpy(a).cuda(), out=o)
    assert rel(o.cpu().numpy()[1], ref) < tol
    clean(p, ("scalar", mode))
p.set_mode(sht.MODE_FP64)
E = inputs.gaussian_alm(L, L, seed=62, nmaps=2)
lv, _ = inputs.lm_arrays(L, L)
E[:, lv < 2] = 0
qu = p.alm2map_spin(torch.from_numpy(np.ascontiguousarray(E[None])).cuda()).cpu().numpy()[0]
q, u = oracle.spin_alm2map_exact(geom, E[0], E[1], L, L)
assert rel(np.concatenate([qu[0], qu[1]]), np.concatenate([q, u])) < 1e-11
eb = p.map2alm_spin(torch.from_numpy(qu[None].copy()).cuda()).cpu().numpy()[0]
clean(p, "spin")
p.set_mlist([0, 7, 64])
p.map2alm(p.alm2map(torch.from_numpy(a).cuda()))
clean(p, "m list")
p.set_mlist(None)
g2 = geometry.gauss_legendre(33, 67)
q2 = sht.Plan(g2, 32, 32, grid=sht.GRID_GAUSS_LEGENDRE)
a2 = inputs.uniform_alm(32, 32, seed=63)
b2 = q2.map2alm(q2.alm2map(torch.from_numpy(a2).cuda())).cpu().numpy()[0]
assert rel(b2, a2[0]) < 1e-12
clean(q2, "gauss-legendre")
x = torch.from_numpy(a).cuda()
y = torch.empty((2, p.npix), dtype=torch.float64, device="cuda")
z = torch.empty((1, q2.nalm), dtype=torch.complex128, device="cuda")
jobs = [batch.Job(p, batch.ALM2MAP, x, y), batch.Job(q2, batch.MAP2ALM, q2.alm2map(torch.from_numpy(a2).cuda()), z)]
pb = batch.PersistentBatch(jobs)
pb.run_eager()
torch.cuda.synchronize()
assert torch.equal(y, p.alm2map(x))
clean(p, "batch")
pb.close()
p.close()
q2.close()
print("checked ok")
'''


def test_checked_build_runs_clean_on_every_entry_point():
    from paper_1106_0159_gb300 import _build
    lib = _build.build(checked=True)
    assert "_lib_check" in lib
    r = subprocess.run([sys.executable, "-c", CHILD, lib, ROOT], capture_output=True, text=True, timeout=1200,
                       cwd=ROOT)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
