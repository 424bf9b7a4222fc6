"""The Rayleigh draw of Eq. 4 as the binning kernel computes it, against FP64.

The kernel takes w_sa = sigma_sa sqrt(-2 ln u), u = (x + 1) / 2^32, with its
own branch-free logarithm (an atanh series on the mantissa, and the integer
complement 2^32 - 1 - x for u >= sqrt(1/2)).  An empty scene makes every bin's
noised value the additive term alone (Eq. 3: P = 0 removes Eq. 5's product),
I~ = (r_c^2 / r_max^2) (1 + 0.5 exp(-phi_c^2 / sigma_phi) w_sa), so w_sa is
recovered from I~ bin by bin and compared with the oracle's FP64 draw from
the same Philox word.  sigma_sa = 2^26 makes the w_sa term dominate the 1 it
is added to, so FP32 rounding of I~ costs only a few units in the last place
of w_sa, even for u within 2^-32 of 1.  Bin b draws word b mod 4 of the
Philox block of counter (b / 4, frame lo, 1, frame hi).  The draws are grouped
by their word:
near 0 (u near 2^-32), near 2^32 - 1 (u near 1) and around 0xB504F333, where
the kernel switches between its two forms of ln u.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import RenderParams, Sonar  # noqa: E402

SIGMA_SA = float(2 ** 26)
RTOL = 2e-6          # about 32 units in the last place of FP32
SEED = 0x9E37_79B9_7F4A_7C15 & 0x7FFF_FFFF_FFFF_FFFF
FRAMES = 16


def test_rayleigh_log_against_fp64():
    son = Sonar(0)
    try:
        mesh = S.Mesh(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.int32))
        sid = son.upload_mesh(mesh)
        spec = S.SensorSpec(np.zeros(3, np.float32), np.eye(3, dtype=np.float32), 8, 1, 1000, 1024,
                            0.2, 0.05, 1.0, 2.0)
        prm = RenderParams(sigma_sa=SIGMA_SA, sigma_sm=0.0, normalise=0)
        theta = son.theta(0.05, 1.0, np.array([0.5], np.float32))
        nr, naz = spec.n_range_bins, spec.n_az_bins
        rmin, rmax = float(np.float32(spec.r_min)), float(np.float32(spec.r_max))
        H = float(np.float32(spec.hfov))
        rc = rmin + (np.arange(nr) + 0.5) * (rmax - rmin) / nr
        pc = -H / 2 + (np.arange(naz) + 0.5) * H / naz
        c = (rc * rc / (rmax * rmax))[:, None]
        pat = (0.5 * np.exp(-pc * pc / prm.sigma_phi))[None, :]
        key = np.array([SEED & 0xFFFFFFFF, SEED >> 32], np.uint32)
        groups = {"near 0": [], "near 2^32-1": [], "around 0xB504F333": [], "all": []}
        for frame in range(FRAMES):
            In = son.render(sid, spec, theta, prm, SEED, frame, fan=False)["noised"]
            torch.cuda.synchronize()
            w_gpu = (In.double().cpu().numpy() / c - 1.0) / pat
            w_ref, _ = O.noise_draws(nr * naz, SEED, frame, SIGMA_SA, 0.0)
            # the additive draw of bin b: word b mod 4 of counter (b / 4, frame, 1, 0)
            ctr = np.zeros((nr * naz // 4, 4), np.uint32)
            ctr[:, 0] = np.arange(nr * naz // 4, dtype=np.uint32)
            ctr[:, 1] = frame
            ctr[:, 2] = 1
            x = O.philox(ctr, key).reshape(-1).astype(np.int64)
            # relative error, on a floor of w_sa = 1 (1.5e-8 sigma_sa): at w_sa = 0 the
            # recovery's own rounding of r_c^2 / r_max^2 leaves about 1e-6
            err = np.abs(w_gpu.ravel() - w_ref) / np.maximum(w_ref, 1.0)
            for name, sel in (("near 0", x < 2 ** 20), ("near 2^32-1", x >= 2 ** 32 - 2 ** 20),
                              ("around 0xB504F333", np.abs(x - 0xB504F333) < 2 ** 20),
                              ("all", np.ones(x.shape, bool))):
                groups[name].append(err[sel])
        report = {}
        for name, parts in groups.items():
            e = np.concatenate(parts)
            assert e.size > 1000, (name, e.size)
            report[name] = (e.size, float(e.max()))
        print("max relative error of the recovered w_sa:", report)
        for name, (n, worst) in report.items():
            assert worst <= RTOL, (name, n, worst)
        st, bits = son.check()
        assert st == 0 and bits == 0
    finally:
        son.close()
