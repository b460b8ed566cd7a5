"""Host-side logic of the benchmark (no GPU): the kernel names it reports for
the library's dispatch, the multigrid cycle's algorithmic bytes, and the 3D
workload generator's shape and mean."""
import numpy as np

import bench
import synth


def test_kernel_names_follow_the_dispatch():
    big, small = 16384 * 16384, 2048 * 2048
    assert bench.kernel_name("f32", 1, big) == "relax1_stream<float,4>"
    assert bench.kernel_name("f64", 1, big) == "relax1_stream<double,2>"
    assert bench.kernel_name("f64", 4, big) == "relaxT_tile<double,4>"
    # the register wavefront from 2^23 cells at depths 3..8
    for tb in range(3, 9):
        assert bench.kernel_name("f32", tb, 1 << 23) == f"relaxR2_f32<{tb}>"
    assert bench.kernel_name("f32", 2, big) == "relaxW2_f32<2>"
    # below 2^23 cells: the one-row wavefront at 6 and 7, the two-row one otherwise
    assert bench.kernel_name("f32", 6, small) == "relaxW_f32<6>"
    assert bench.kernel_name("f32", 8, small) == "relaxW2_f32<8>"


def test_multigrid_algorithmic_bytes():
    """Elements per cell on every level but the coarsest (levels halve while
    the extent is a multiple of 4): 8.75 in FP32 (the interpolation inside the
    post-smoothing launch), 10.75 in FP64 (a pass of its own)."""
    for n, es in ((16384, 4), (256, 8), (96, 4)):
        cells, m = 0, n
        while m % 4 == 0:
            cells += m * m
            m //= 2
        assert bench.mg_algo_bytes(n, es) == es * (8.75 if es == 4 else 10.75) * cells
    # 16384^2 FP32: 12.53 GB per V(2,2) cycle (4/3 of the finest level's 35 B per cell)
    assert abs(bench.mg_algo_bytes(16384, 4) / 1e9 - 12.53) < 0.01


def test_field3_workload():
    r = synth.field3_rho(32, nmodes=4, kmax=8, seed=1)
    assert r.shape == (32, 32, 32)
    assert abs(r.mean()) < 1e-12
    r2 = synth.field3_rho(32, nmodes=4, kmax=8, seed=1)
    assert np.array_equal(r, r2)  # seeded


def test_digest_is_short_and_complete():
    """The digest closing the bench line carries every block's headline figure
    in well under the 1500 characters a reader of the line's tail keeps."""
    import json
    v = {"GLUP_s": 1.0, "hbm_frac": 0.5, "ms_per_step": 1.0}
    line = {
        "value": 2572.2, "roofline": {"frac": 0.594},
        "variants": {k: dict(v) for k in ("f32_t1", "f32_t2", "f32_t4", "f32_t8")},
        "rbsor": {"f32": v, "f64": v},
        "multigrid": {"f32": {"ms_per_cycle": 3.2}, "f64": {"ms_per_cycle": 37.0}},
        "relax3d": {"f32": v, "f64": v},
        "batched": {"ms": 347.0},
        "time_to_1e-8": {"plain_f64": {"ms": 278.0}, "mixed": {"ms": 86.0}, "grid": 256},
        "refine_8192": {k: {"cycles": 3, "wall_s": 1.0, "rel_resid": 1e-11}
                        for k in ("literal", "noise_free", "mg_f64_literal")},
        "euler": {"f64": {"Gcell_s": 1.0, "hbm_frac": 0.8}, "f32": {"Gcell_s": 2.0, "hbm_frac": 0.8}},
        "e2e": {"value": 1500.0},
    }
    for k in ("f64_t1", "f64_t2", "f64_t4", "f64_t8"):
        line["variants"][k] = dict(v, fp64_pipe_frac=0.7)
    d = bench.digest(line)
    assert d["T"]["f64_t4"] == [1.0, 0.7] and d["T"]["f32_t8"] == [1.0, 0.5]
    assert d["c3"]["noise_free"] == [3, 1.0, 1e-11]
    assert d["euler"]["f32"] == [2.0, 0.8]
    assert len(json.dumps(d)) < 1000


def test_batch_fp64_bound_operations():
    """FP64 instances count 6 operations per update in shared memory and 5
    banded; FP32 classes do not count."""
    classes = {"f64:64x64@c2": {"count": 3, "mode": "whole"},
               "f64:512x256@c2s": {"count": 2, "mode": "banded"},
               "f32:1024x1024@c2": {"count": 7, "mode": "banded_t"}}
    assert bench.batch_fp64_ops(classes) == 3 * 64 * 64 * 6 + 2 * 512 * 256 * 5
    assert bench.batch_fp64_ops({}) == 0

