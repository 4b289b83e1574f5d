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
