"""Distribution-level parity of the 64-qubit noisy workload (8x8 grid, p = 2):
the sample means of Z_u Z_v on the eight corner edges against their exact
values from the oracle's light-cone density matrix (Sec. 3: Alg. 2 samples
the diagonal of the noisy circuit's density matrix), on both engines, at the
workload's own noise and with the noise raised until it moves the correlators
by many standard errors."""
import numpy as np
import pytest

import workloads as W
from oracle import lightcone as LC

from tests.test_gpu_parity import run_gpu

pytestmark = pytest.mark.gpu

SPLIT3 = 0                 # PW_GEMM_SPLIT3 of include/pw.h
ONCHIP, HBM = 1, 2         # PW_ENGINE_* of include/pw.h
CORNERS = [(0, 1), (0, 8), (6, 7), (7, 15), (48, 56), (56, 57), (55, 63), (62, 63)]


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_24218_gb300 as mod
    mod.load_library()
    return mod


def _zz_means(bits):
    z = 1.0 - 2.0 * bits.astype(np.float64)
    return np.array([np.mean(z[:, u] * z[:, v]) for u, v in CORNERS])


@pytest.mark.parametrize("noise,engine", [((0.03, 0.05), ONCHIP), ((0.03, 0.05), HBM), ((1e-3, 1e-3), HBM)])
def test_corner_correlators_match_the_density_matrix(pw, noise, engine):
    depol2, ad = noise
    spec = W.grid_8x8_p2_noisy(depol2=depol2, ad_gamma=ad)
    N = 1 << 19
    opts = dict(engine=engine, gemm=SPLIT3) if engine == HBM else dict(engine=engine)
    g = run_gpu(pw, spec, N, seed=31337, trace=False, **opts)
    assert g["stats"]["zero_mass"] == 0
    got = _zz_means(g["bits"])
    want = np.array([LC.zz(spec, u, v) for u, v in CORNERS])
    se = np.sqrt((1.0 - want ** 2) / N)
    assert np.all(np.abs(got - want) < 5 * se), (got, want, se)
    if depol2 > 0.01:
        # the test sees the noise: the noiseless correlators are far off
        clean = LC.zz(W.grid_8x8_p2_noisy(depol2=0.0, ad_gamma=0.0), 0, 1)
        assert np.all(np.abs(clean - want) > 10 * se)
        assert np.all(np.abs(clean - got) > 5 * se)
