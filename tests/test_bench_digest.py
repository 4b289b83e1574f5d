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
    # mixed precision, fused sort gather: 2 x (3 FP64 coordinates + 3 FP32
    # momenta) + permutation, sorted id and id write = 84 B per grain; gas
    # (4 x FP32) + int64 deposit (4 x 8) = 48 B per zone
    from paper_1908_10793_gb300 import inputs as I
    w = I.sbox3d("small")
    total, per_grain, per_zone = bench.algorithmic_bytes(w, 4, fused_gather=True)
    assert (per_grain, per_zone) == (84, 48)
    assert total == 84 * w.ngrains + 48 * w.ncell
    # the bench workload: 16.8M grains and 2.1M zones -> 1.51 GB per launch
    assert 84 * 16_777_216 + 48 * 128 ** 3 == 1_509_949_440
