"""bench.py ties the committed ncu figures of the step kernel to a digest of
its sources; the digest follows the code, not the comments."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reader(edit):
    def read(f):
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        return edit(f, text)
    return read


def test_digest_ignores_comments_and_layout_but_not_code():
    base = bench.source_digest()
    assert bench.source_digest(read=_reader(lambda f, t: t)) == base
    comment = _reader(lambda f, t: t + "\n// a note\n/* another\n   note */\n" if f.endswith(".cuh") else t)
    layout = _reader(lambda f, t: t.replace("\n", "\n\n") if f.endswith("dust_slab.cuh") else t)
    code = _reader(lambda f, t: t.replace("kSlabCap = 128", "kSlabCap = 64") if f.endswith("dust_slab.cuh") else t)
    assert bench.source_digest(read=comment) == base
    assert bench.source_digest(read=layout) == base
    assert bench.source_digest(read=code) != base


def test_code_only_keeps_string_and_character_literals():
    src = 'int a = 1; // c\n/* x\n y */ const char *s = "a // b /* c */"; char q = \'"\';'
    assert bench._code_only(src) == 'int a = 1; const char *s = "a // b /* c */"; char q = \'"\';'


def test_algorithmic_bytes_of_the_mixed_step():
    # mixed precision: 2 x (3 FP64 coordinates + 3 FP32 momenta) = 72 B per
    # grain; gas (4 x FP32) + int64 deposit (4 x 8) = 48 B per zone; at 8
    # grains per zone 78 B per grain.  The zone sort's permutation and id
    # traffic (12 B per grain in the step kernel) is reported apart.
    from paper_1908_10793_gb300 import inputs as I
    w = I.sbox3d("small")
    total, per_grain, per_zone = bench.algorithmic_bytes(w, 4)
    assert (per_grain, per_zone) == (72, 48)
    assert total == 72 * w.ngrains + 48 * w.ncell
    assert total == 78 * w.ngrains
    # the bench workload: 16.8M grains and 2.1M zones -> 1.309 GB per launch
    assert 72 * 16_777_216 + 48 * 128 ** 3 == 1_308_622_848

    class KT:
        sort_ms, sort_launches = 4.0, 12
    so = bench.sort_overhead(w, KT, 2)
    assert so["step_kernel_bytes_per_grain"] == 12
    assert so["step_kernel_bytes_per_launch"] == 12 * w.ngrains
    assert so["sort_kernels_ms_per_step"] == 2.0 and so["sort_kernel_launches_per_step"] == 6
