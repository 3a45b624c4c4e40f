"""Host checks of bench.py's roofline bookkeeping (no GPU).

The bench reports, for the dominant kernel, algorithmic bytes over the
kernel's event time and DRAM traffic scaled from an ncu capture.  Both are
keyed by the launch names the library gives its kernels, so a renamed launch
would silently drop them: every traffic entry must name a launch the library
makes, and every heavy launch must have an algorithmic byte count.
"""
import importlib.util
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the bench workload: B 1, width 20, 128^3 x 32, modes 12/12/8/8
DD = {"B": 1, "Ci": 20, "Co": 20, "Nx": 128, "Ny": 128, "Nz": 128, "Nt": 32,
      "Jx": 24, "Jy": 24, "Jz": 16, "Jt": 8}
GRID = 4 * 1 * 20 * 128 ** 3 * 32  # bytes of one FP32 activation tensor


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def launch_names():
    names = set()
    for p in glob.glob(os.path.join(ROOT, "paper_2211_12709_gb300", "csrc", "*.cu")):
        names.update(re.findall(r'"(fno_[a-z0-9_]+)"', open(p).read()))
    return names


def test_traffic_entries_name_launches_of_the_library():
    b = _bench()
    names = launch_names()
    assert "fno_da_saved" in names and "fno_epi_fwd_train_mma_bf16x3" in names
    assert "fno_da_tz_bf16x3" in names
    for key in b.TRAFFIC_PER_UNIT:
        assert key in names, key


def test_every_heavy_launch_has_algorithmic_bytes():
    b = _bench()
    heavy = [n for n in launch_names()
             if n.startswith(("fno_epi_fwd", "fno_epi_da", "fno_epi_dx", "fno_fwd_tz", "fno_da_saved",
                              "fno_da_tz", "fno_mix", "fno_synth_t", "fno_pw_add"))]
    assert len(heavy) >= 25
    for n in heavy:
        nbytes, _ = b.algorithmic(n, DD)
        # every one moves at least one activation tensor, except the mixing
        # kernels, which move the weights and the kept spectra
        assert nbytes and nbytes > (0 if n.startswith("fno_mix") else GRID), n


def test_training_forward_counts_the_derivative_store():
    b = _bench()
    train, _ = b.algorithmic("fno_epi_fwd_train_mma_bf16x3", DD)
    plain, _ = b.algorithmic("fno_epi_fwd_mma_bf16x3", DD)
    assert train - plain == GRID
    # the dA pass reads x, dz and GELU'(A) and writes dA; the fused pass also
    # writes the t,z spectrum of dA and adds the t,z DFT's flops
    assert b.algorithmic("fno_da_saved", DD)[0] == 4 * GRID
    fb, ff = b.algorithmic("fno_da_tz_bf16x3", DD)
    tb, tf = b.algorithmic("fno_fwd_tz_mma_bf16x3", DD)
    assert fb == 4 * GRID + (tb - GRID)
    assert ff == b.algorithmic("fno_da_saved", DD)[1] + tf


def test_roofline_fraction_is_algorithmic_bytes_over_time_over_peak():
    b = _bench()
    pk = {"hbm_gbs": 6754.1, "bf16_tflops": 1929.9, "sm_max_mhz": 2070.0, "src": "measured"}
    nbytes = b.algorithmic("fno_da_tz_bf16x3", DD)[0]
    r = b.roofline_of("fno_da_tz_bf16x3", 4.81, DD, pk, "bf16x3")
    achieved = nbytes / 4.81e-3 / 1e9
    assert r["bound"] == "hbm"
    assert abs(r["achieved"] - achieved) < 0.5
    assert abs(r["frac"] - achieved / 6754.1) < 1e-3
    assert r["traffic"] is not None and abs(r["traffic"] / nbytes - 1) < 0.05


def test_synthesis_path_counts_its_tensors():
    # at the CO2 paper grid (B 1, width 20, 262 x 118 x 64 x 86, modes 26/12/6/8)
    b = _bench()
    dd = {"B": 1, "Ci": 20, "Co": 20, "Nx": 262, "Ny": 118, "Nz": 64, "Nt": 86,
          "Jx": 52, "Jy": 24, "Jz": 12, "Jt": 8}
    grid = 4 * 20 * 262 * 118 * 64 * 86
    v = 8 * 20 * 262 * 118 * 64 * 8  # the inverse z stage's output, complex64
    assert b.algorithmic("fno_pw_add_fwd", dd)[0] == 4 * grid
    assert b.algorithmic("fno_pw_add_dx", dd)[0] == 2 * grid
    sb, sf = b.algorithmic("fno_synth_t_bf16x3", dd)
    assert sb == v + 3 * grid // 2
    assert sf == 20 * 262 * 118 * 64 * 86 * 8 * 4  # (re, im) products per point, mode and channel
    pk = {"hbm_gbs": 6685.5, "bf16_tflops": 1942.4, "sm_max_mhz": 2070.0, "src": "measured"}
    assert b.roofline_of("fno_synth_t_bf16x3", 5.148, dd, pk, "bf16x3")["bound"] == "hbm"
    r = b.roofline_of("fno_pw_add_fwd", 13.985, dd, pk, "bf16x3")
    assert r["bound"] == "hbm" and abs(r["frac"] - 4 * grid / 13.985e-3 / 1e9 / 6685.5) < 1e-3
