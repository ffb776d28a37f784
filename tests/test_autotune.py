"""Host logic of the screen-schedule autotuner: cache keys, lookups and the
deepest-section size it keys on (no GPU needed)."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2106_12942_b300 import autotune as A  # noqa: E402


def test_deepest_section_size_matches_floor_halving():
    # the library splits at floor(h/2): the first half is the smaller one
    assert A.deepest_section_px(1024, 1024, 5) == 64 * 64
    assert A.deepest_section_px(2048, 2048, 6) == 64 * 64
    assert A.deepest_section_px(145, 145, 3) == 37 * 37     # 145 -> 72 | 73 -> 36 | 37
    assert A.deepest_section_px(7, 5, 1) == 35


def test_bucket_and_key():
    assert [A.bucket(n) for n in (1, 2, 3, 4096, 4097)] == [1, 2, 4, 4096, 8192]
    assert A.cache_key(224, 4096) == "sm_103a/B224/n4096"
    assert A.cache_key(224, 3000) == A.cache_key(224, 4096)


def test_lookup_reads_the_stored_choice(tmp_path):
    path = str(tmp_path / "cache.json")
    assert A.lookup(224, 4096, path=path) == {}
    json.dump({A.cache_key(224, 4096): {"screen_group": 7, "screen_ms": {"4": 1.0, "7": 0.9}},
               A.cache_key(128, 1024): {"screen_pair": 1, "screen_group": 2}}, open(path, "w"))
    assert A.lookup(224, 4096, path=path) == {"screen_group": 7, "screen_pair": 0}    # entry without a form
    assert A.lookup(128, 1024, path=path) == {"screen_group": 2, "screen_pair": 1}
    assert A.lookup(128, 4096, path=path) == {}
    assert A.lookup(64, 1024, path=path) == {}
