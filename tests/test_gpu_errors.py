"""Failure paths of the C-ABI on the GPU: argument validation, state errors, injected
allocation failure, bounded device waits that give up.  None of these faults or hangs the
GPU: timeouts come from waits with a short poll limit, never from a trap or a bad address."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2210_04184_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2210_04184_gb300 import build as _build  # noqa: E402
from paper_2210_04184_gb300 import fuse  # noqa: E402
from paper_2210_04184_gb300.fuse import Fusion, FuseError  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()


def _p(**kw):
    base = dict(H=40, W=40, L_l=6, L_h=2, L_s=3, d=4, blur_size=5, blur_sigma=1.0, K=1, S=2,
                lam1=1.0, lam2=1e-2, rho=5e-2, h=0.3, seed=3)
    base.update(kw)
    return synth.make_problem(**base)


def _t(a):
    return torch.tensor(a, dtype=torch.float32, device="cuda")


def test_init_rejects_bad_arguments():
    p = _p()
    g = fuse.fuse_geometry(p.H, p.W, p.L_l, p.L_h, p.L_s, p.L_h)
    with pytest.raises(FuseError) as e:
        fuse.fuse_init(g, p.blur, p.d, p.R, p.E, p.K, p.S, 1.0, 1e-2, -1.0, 0.3, fuse.FUSE_F32, fuse.FUSE_F32)
    assert e.value.status == fuse.FUSE_EINVAL
    with pytest.raises(FuseError) as e:
        fuse.fuse_init(g, np.ones((4, 4)), p.d, p.R, p.E, p.K, p.S, 1.0, 1e-2, 0.1, 0.3, fuse.FUSE_F32,
                       fuse.FUSE_F32)
    assert e.value.status == fuse.FUSE_EINVAL          # even blur size
    g2 = fuse.fuse_geometry(p.H, p.W, p.L_l, p.L_h, p.L_s + 1, p.L_h)
    with pytest.raises(FuseError) as e:
        fuse.fuse_init(g2, p.blur, p.d, p.R, None, p.K, p.S, 1.0, 1e-2, 0.1, 0.3, fuse.FUSE_F32, fuse.FUSE_F32)
    assert e.value.status == fuse.FUSE_EINVAL          # E = I needs L_s = L_l


def test_solve_before_weights_is_a_state_error():
    p = _p()
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    with pytest.raises(FuseError) as e:
        f.solve(_t(p.Yl), _t(p.Yh), 3)
    assert e.value.status == fuse.FUSE_ESTATE
    with pytest.raises(FuseError) as e:
        f.solve(_t(p.Yl), _t(p.Yh), -1)
    assert e.value.status == fuse.FUSE_EINVAL
    f.close()


def test_bad_option_keeps_previous_setting():
    p = _p()
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    with pytest.raises(FuseError):
        f.set_option(fuse.FUSE_OPT_LATENT_STAGES, 1000)
    fuse.fuse_reset_error(f.ctx)
    f.weights(_t(p.Yh))
    X, _ = f.solve(_t(p.Yl), _t(p.Yh), 3)
    f.sync()
    assert torch.isfinite(X).all()


def test_injected_allocation_failure_returns_enomem():
    code = (
        "import os, sys; sys.path.insert(0, %r)\n"
        "from paper_2210_04184_gb300 import synth, fuse\n"
        "p = synth.make_problem(H=40, W=40, L_l=6, L_h=2, L_s=3, d=4, blur_size=5, K=1, S=2, seed=3)\n"
        "g = fuse.fuse_geometry(40, 40, 6, 2, 3, 2)\n"
        "for k in range(0, 12):\n"
        "    os.environ['FUSE_FAULT_ALLOC'] = str(k)\n"
        "    try:\n"
        "        fuse.fuse_init(g, p.blur, 4, p.R, p.E, 1, 2, 1.0, 1e-2, 0.05, 0.3, 0, 0)\n"
        "        raise SystemExit('no failure injected at %%d' %% k)\n"
        "    except fuse.FuseError as e:\n"
        "        assert e.status == fuse.FUSE_ENOMEM, e\n"
        "print('ok')\n" % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_selftest_bounded_wait_reports_timeout():
    p = _p()
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    fuse.fuse_selftest(f.ctx, 1)
    # the context stays usable
    f.weights(_t(p.Yh))
    X, _ = f.solve(_t(p.Yl), _t(p.Yh), 4)
    f.sync()
    assert torch.isfinite(X).all()


def test_latent_short_wait_limit_is_bounded_and_recoverable():
    # One poll per barrier wait (each poll may suspend for a hardware time window): the
    # pipelined latent pass either still sees every copy land (bit-identical result) or gives up
    # on a wait and fuse_sync reports FUSE_ETIMEOUT; either way it finishes and the context is
    # usable again after fuse_reset_error.
    p = _p(H=48, W=64, K=2, S=3, L_l=8, L_h=3, L_s=4)
    ref = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    ref.weights(_t(p.Yh))
    a, _ = ref.solve(_t(p.Yl), _t(p.Yh), 3)
    ref.sync()
    f = Fusion.from_problem(p, dtype="f32", wdtype="f32")
    f.weights(_t(p.Yh))
    f.set_option(fuse.FUSE_OPT_WAIT_LIMIT, 1)
    b, _ = f.solve(_t(p.Yl), _t(p.Yh), 3)
    try:
        f.sync()
        assert torch.equal(a, b)
    except FuseError as e:
        assert e.status == fuse.FUSE_ETIMEOUT
        fuse.fuse_reset_error(f.ctx)
    f.set_option(fuse.FUSE_OPT_WAIT_LIMIT, 1 << 22)
    b, _ = f.solve(_t(p.Yl), _t(p.Yh), 3)
    f.sync()
    assert torch.equal(a, b)
