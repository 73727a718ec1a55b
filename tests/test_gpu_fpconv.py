"""The integer-pipe FP32 <-> FP64 conversions of the FP32-storage kernels
(rlbm_convert_f32_f64) against the hardware conversions, on edge values:
exact ties, the largest and smallest normals, denormals, infinities, NaN,
signed zeros, and random bit patterns."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04502_gb300 import build, rlbm
    build.build()
    return rlbm


def _run(rl, f, d):
    import torch
    tf = torch.tensor(f, dtype=torch.float32, device="cuda")
    td = torch.tensor(d, dtype=torch.float64, device="cuda")
    od = torch.empty(len(f), dtype=torch.float64, device="cuda")
    of = torch.empty(len(d), dtype=torch.float32, device="cuda")
    rc = rl.lib().rlbm_convert_f32_f64(tf.data_ptr(), od.data_ptr(), len(f), td.data_ptr(), of.data_ptr(), len(d),
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return tf, td, od, of


def test_float_to_double_is_exact_for_normals_and_flushes_denormals(rl):
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, np.finfo(np.float32).max, np.finfo(np.float32).tiny,
                        -np.finfo(np.float32).tiny, 1e-40, -3e-42, 1.0, -2.5], dtype=np.float32)
    f = np.concatenate([f, special])
    tf, _, od, _ = _run(rl, f, np.zeros(0))
    hw = tf.double().cpu().numpy()
    got = od.cpu().numpy()
    normal = np.isfinite(f) & (np.abs(f) >= np.finfo(np.float32).tiny)
    assert np.array_equal(got[normal], hw[normal])
    den = np.isfinite(f) & (np.abs(f) < np.finfo(np.float32).tiny)
    assert np.all(got[den] == 0.0) and np.array_equal(np.signbit(got[den]), np.signbit(f[den]))
    assert np.array_equal(np.isnan(got), np.isnan(f))
    inf = np.isinf(f)
    assert np.array_equal(got[inf], hw[inf])


def test_double_to_float_rounds_to_nearest_with_ties_away_from_zero(rl):
    rng = np.random.default_rng(2)
    d = rng.standard_normal(200000) * np.exp(rng.uniform(-80, 80, 200000))
    # exact ties: halfway between two adjacent floats
    base = rng.standard_normal(2000).astype(np.float32)
    up = np.nextafter(base, np.float32(np.inf))
    ties = (base.astype(np.float64) + up.astype(np.float64)) / 2
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38, 1e39, -1e39, 1e-39, -1e-44,
                        1.1754943508222875e-38, 1.0, -1.0 - 2 ** -30])
    d = np.concatenate([d, ties, special])
    _, td, _, of = _run(rl, np.zeros(0, dtype=np.float32), d)
    hw = td.float().cpu().numpy()                     # round to nearest even
    got = of.cpu().numpy()
    tie = np.zeros(len(d), dtype=bool)
    tie[200000:202000] = True
    small = np.isfinite(d) & (np.abs(d) < np.finfo(np.float32).tiny) & ~np.isnan(d)
    ok = np.isfinite(hw) & ~tie & ~small
    assert np.array_equal(got[ok], hw[ok])
    # ties go away from zero
    away = np.where(np.abs(base) < np.abs(up), up, base)
    assert np.array_equal(got[tie], away)
    # below the smallest normal: signed zero
    assert np.all(got[small] == 0.0) and np.array_equal(np.signbit(got[small]), np.signbit(d[small]))
    # overflow and infinities keep their sign, NaN stays NaN
    big = np.isfinite(d) & (np.abs(d) > 3.4028235677973366e38)
    assert np.all(np.isinf(got[big])) and np.array_equal(np.signbit(got[big]), np.signbit(d[big]))
    assert np.array_equal(np.isnan(got), np.isnan(d))
    assert np.array_equal(got[np.isinf(d)], hw[np.isinf(d)])
