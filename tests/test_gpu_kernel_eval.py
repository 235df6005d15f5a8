"""The device kernel functions (Sec. 6) against extended-precision references: the
table-driven exponential (Tang's method) inside the EXP, GAUSS and MATERN32 kernels stays
within two units in the last place of the exact value, and within three of CUDA's own
exp; the exponent's arguments are formed exactly as the device forms them."""
import numpy as np
import pytest
import torch

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def ulps(got, ref):
    """|got - ref| in units in the last place of the double nearest to ref."""
    refd = ref.astype(np.float64)
    return np.abs(got.astype(np.longdouble) - ref) / np.spacing(np.abs(refd)).astype(np.longdouble)


def r2_samples(ell):
    rng = np.random.default_rng(0)
    # arguments -sqrt(r2)/ell spread over [-700, 0], plus the points where the reduction
    # switches table entries (odd multiples of ln2/128) and the edges
    x = np.concatenate([-rng.uniform(0, 700, 200000), -rng.uniform(0, 1, 50000),
                        -(np.arange(1, 2000) * 2 - 1) * np.log(2) / 128,
                        [0.0, -1e-300, -5e-324, -1e-12, -699.999, -700.0]])
    return (x * ell) ** 2


@pytest.mark.parametrize("ell", [1.0, 0.37, 3.0])
def test_exp_kernel_within_two_ulps(ell):
    api = need_gpu()
    r2 = r2_samples(ell)
    got = api.kernel_eval("exp", ell, r2).cpu().numpy()
    x = -np.sqrt(r2) * (1.0 / ell)          # the device's argument, bit for bit
    ref = np.exp(x.astype(np.longdouble))
    assert ulps(got, ref).max() <= 2.0
    cuda = torch.exp(torch.from_numpy(x).cuda()).cpu().numpy()
    assert (np.abs(got - cuda) / np.spacing(np.abs(cuda))).max() <= 3.0
    assert got[r2 == 0.0].min() == 1.0 and got[r2 == 0.0].max() == 1.0


def test_gauss_and_matern_kernels():
    api = need_gpu()
    ell = 0.8
    r2 = r2_samples(1.0) * 0.0005          # Gaussian arguments -r2/ell^2 down to ~ -380
    inv = 1.0 / ell
    got = api.kernel_eval("gauss", ell, r2).cpu().numpy()
    ref = np.exp((-r2 * (inv * inv)).astype(np.longdouble))
    assert ulps(got, ref).max() <= 2.0
    r2m = r2_samples(1.0) / 3.0
    got = api.kernel_eval("matern32", ell, r2m).cpu().numpy()
    t = 1.7320508075688772 * np.sqrt(r2m) * inv
    ref = (1.0 + t.astype(np.longdouble)) * np.exp(-t.astype(np.longdouble))
    ok = ref > np.longdouble(1e-300)
    assert ulps(got[ok], ref[ok]).max() <= 4.0


def test_below_the_table_range_and_imq():
    api = need_gpu()
    r2 = np.array([700.5, 720.0, 745.0, 800.0, 1e6]) ** 2
    got = api.kernel_eval("exp", 1.0, r2).cpu().numpy()
    cuda = torch.exp(-torch.from_numpy(np.sqrt(r2)).cuda()).cpu().numpy()
    assert np.array_equal(got, cuda)
    r2 = np.random.default_rng(1).uniform(0, 100, 10000)
    got = api.kernel_eval("imq", 0.5, r2).cpu().numpy()
    ref = 1.0 / np.sqrt(1.0 + r2.astype(np.longdouble) * 4.0)
    assert ulps(got, ref).max() <= 2.0


def test_rejects_rpy_and_host_arrays():
    api = need_gpu()
    from paper_2011_07632_gb300 import native as N
    with pytest.raises(N.SpdhssError):
        api.kernel_eval("rpy", 1.0, np.ones(4))
    r2 = np.ones(4)
    out = np.zeros(4)
    st = N.lib().spdhss_kernel_eval(N.KernelDesc(N.KERNELS["exp"], 1.0, 0.0),
                                    r2.ctypes.data, out.ctypes.data, 4, None)
    assert st != 0
