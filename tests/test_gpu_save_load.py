"""Checkpoint and resume (pft_save / pft_load): a complex Langevin run interrupted by a
save and continued in a fresh context reproduces the uninterrupted run bit for bit
(fields, noise key and counter restored); the box of a variable-cell run comes back;
a checkpoint of another system, a missing, foreign, truncated or corrupted file and a
save before the fields are set are refused with the documented status."""
import os

import numpy as np
import pytest

from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu

FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _cl_fields(n, seed):
    rng = np.random.default_rng(seed)
    wp = 0.05 * (rng.normal(size=n) + 1j * rng.normal(size=n))
    wm = 0.2 * (rng.normal(size=n) + 1j * rng.normal(size=n))
    return wp, wm


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_cl_run_resumes_bit_for_bit(tmp_path, prec):
    n, L, Ns, fA, chiN, C, dt = (16, 8, 12), (4.0, 2.0, 3.0), 12, 0.3, 20.0, 50.0, 0.01
    wp, wm = _cl_fields(n, 5)
    path = str(tmp_path / "run.ckpt")
    with pft.System(n, L, Ns, fA, chiN, C, CL, prec, seed=1234, instance=3) as s:
        s.set_fields(wp, wm)
        for _ in range(3):
            s.solve()
            s.field_step(dt)
        s.save(path)
        for _ in range(2):
            s.solve()
            s.field_step(dt)
        s.solve()
        ref_p, ref_m = s.get_fields()
        ref_H = s.observables()["H"]
    # a context with another noise key: the checkpoint's key and counter take over
    with pft.System(n, L, Ns, fA, chiN, C, CL, prec, seed=99, instance=0) as s:
        s.set_fields(np.zeros(n, complex), np.zeros(n, complex))
        s.load(path)
        for _ in range(2):
            s.solve()
            s.field_step(dt)
        s.solve()
        gp, gm = s.get_fields()
        H = s.observables()["H"]
    assert np.array_equal(gp, ref_p) and np.array_equal(gm, ref_m)
    assert H == ref_H
    assert not os.path.exists(path + ".tmp")


def test_precision_may_differ_and_box_is_restored(tmp_path):
    n, L, Ns, fA, chiN = (8, 8, 16), (2.0, 2.0, 4.0), 10, 0.4, 15.0
    rng = np.random.default_rng(2)
    wp, wm = rng.normal(0, 0.3, n), rng.normal(0, 1.0, n)
    path = str(tmp_path / "cell.ckpt")
    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        s.set_box((2.1, 1.9, 4.2))
        s.save(path)
        s.solve()
        Q64 = s.observables()["Q"].real
    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP32) as s:
        s.load(path)
        assert pft.pft_get_box(s.h) == (2.1, 1.9, 4.2)
        gp, gm = s.get_fields()
        assert np.array_equal(gp, wp) and np.array_equal(gm, wm)
        s.solve()
        assert abs(s.observables()["Q"].real - Q64) <= 2e-5 * Q64


def test_edwards_checkpoint_round_trip(tmp_path):
    n, L, Ns = (8, 8, 8), (2.0, 2.0, 2.0), 8
    w = np.random.default_rng(4).normal(0, 0.5, n)
    path = str(tmp_path / "edw.ckpt")
    kw = dict(arch=pft.PFT_ARCH_EDWARDS, B=2.0)
    with pft.System(n, L, Ns, 0.5, 1.0, 5.0, SCFT, FP64, **kw) as s:
        s.set_fields(w)
        s.save(path)
    # one field of M float64 after the 128-byte preamble, then the hash
    assert os.path.getsize(path) == 8 + 4 + 4 + 112 + w.size * 8 + 8
    with pft.System(n, L, Ns, 0.5, 1.0, 5.0, SCFT, FP64, **kw) as s:
        s.load(path)
        g, _ = s.get_fields()
        assert np.array_equal(g, w)


def test_refusals(tmp_path):
    n, L, Ns, fA, chiN = (8, 8, 8), (2.0, 2.0, 2.0), 8, 0.5, 15.0
    rng = np.random.default_rng(3)
    wp, wm = rng.normal(0, 0.3, n), rng.normal(0, 1.0, n)
    good = str(tmp_path / "good.ckpt")

    def status(f):
        with pytest.raises(pft.PftError) as ei:
            f()
        return ei.value.status

    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP64) as s:
        assert status(lambda: s.save(good)) == pft.PFT_ERR_STATE
        s.set_fields(wp, wm)
        s.save(good)
        assert status(lambda: s.load(str(tmp_path / "missing.ckpt"))) == pft.PFT_ERR_IO
        assert status(lambda: s.save(str(tmp_path / "no_such_dir" / "x.ckpt"))) == pft.PFT_ERR_IO
        raw = open(good, "rb").read()
        for name, data in (("foreign", b"NOTACKPT" + raw[8:]), ("truncated", raw[:-9]), ("long", raw + b"\0"),
                           ("flipped", raw[:200] + bytes([raw[200] ^ 1]) + raw[201:])):
            p = str(tmp_path / f"{name}.ckpt")
            open(p, "wb").write(data)
            assert status(lambda: s.load(p)) == pft.PFT_ERR_IO, name
        # the refused loads left the context as it was
        gp, gm = s.get_fields()
        assert np.array_equal(gp, wp) and np.array_equal(gm, wm)
    for other in (dict(n=(8, 8, 16)), dict(Ns=9), dict(chiN=14.0), dict(fA=0.4), dict(kind=CL)):
        kw = dict(n=n, L=L, Ns=Ns, fA=fA, chiN=chiN, C=1.0, kind=SCFT, precision=FP64)
        kw.update(other)
        with pft.System(**kw) as s:
            assert status(lambda: s.load(good)) == pft.PFT_ERR_ARG, other
