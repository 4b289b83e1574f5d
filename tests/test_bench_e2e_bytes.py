"""The end-to-end leg's declared host-link bytes per step equal the sizes of
the host arrays it copies (the dtypes the C calls take): grains in and out,
the gas in, the deposit out."""
import numpy as np

import bench


def _arrays(ng, ncell, v32):
    vdt = np.float32 if v32 else np.float64
    ins = [np.empty(ng) for _ in range(3)] + [np.empty(ng, vdt) for _ in range(3)] + \
          [np.empty(ncell) for _ in range(4)]
    outs = [np.empty(ng) for _ in range(3)] + [np.empty(ng, vdt) for _ in range(3)] + \
           [np.empty(ng, np.int64), np.empty((ncell, 4), np.int64)]
    return sum(a.nbytes for a in ins), sum(a.nbytes for a in outs)


def test_e2e_bytes_match_the_copied_arrays():
    for ng, ncell in ((1000, 64), (4096, 4096), (123457, 2197)):
        for v32 in (True, False):
            assert bench.e2e_bytes_per_step(ng, ncell, v32=v32) == _arrays(ng, ncell, v32)


def test_e2e_bytes_of_the_bench_workload():
    # 128^3 zones, 16,777,216 grains: 0.67 GB in and 0.81 GB out with float32
    # velocities, 0.87 / 1.01 GB with float64
    assert bench.e2e_bytes_per_step(16777216, 128 ** 3, v32=True) == (671088640, 805306368)
    assert bench.e2e_bytes_per_step(16777216, 128 ** 3, v32=False) == (872415232, 1006632960)
