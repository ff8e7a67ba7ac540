"""The all-cores (OpenMP) build of the oracle, used only for the CPU timing,
computes exactly what the plain build does: it only spreads independent
meshes, pixel rows, sources and stamps over threads."""
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys, numpy as np
sys.path[:0] = [%r]
import oracle, synth
oracle.use_openmp(4)
img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0, flux=(3.0, 4.5))
oc = oracle.catalog(img, mesh=32)
st, _ = synth.moffat_stamps(64, seed=4000)
fit = oracle.psf_fit(st)
np.savez(sys.argv[1], sub=oc["sub"], labels=oc["labels"], x=oc["x"], y=oc["y"], flux=oc["flux"],
         bkg=oc["bkg"], params=fit["params"], chi2=fit["chi2"])
"""


def test_openmp_build_matches_plain_build(orc, tmp_path):
    out = tmp_path / "omp.npz"
    subprocess.run([sys.executable, "-c", _CHILD % ROOT, str(out)], check=True, timeout=300)
    r = np.load(out)
    img, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0, flux=(3.0, 4.5))
    oc = orc.catalog(img, mesh=32)
    st, _ = synth.moffat_stamps(64, seed=4000)
    fit = orc.psf_fit(st)
    for k in ("sub", "labels", "x", "y", "flux", "bkg"):
        assert np.array_equal(r[k], oc[k]), k
    assert np.array_equal(r["params"], fit["params"]) and np.array_equal(r["chi2"], fit["chi2"])
