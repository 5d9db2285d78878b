"""The autotuner's cache on CPU: leiden_tuning_lookup (the library's JSON
reader and nearest-class selection), the defaults and range checks, the
Python class function and the cache merge. No device work."""
import json
import os
import math

import pytest

import paper_2312_13936_gb300 as lg
from paper_2312_13936_gb300 import tune

GPU = "NVIDIA GB300"


def _entry(heavy, ln, lm, **shape):
    e = {"gpu": GPU, "heavy_tailed": heavy, "log2_vertices": ln, "log2_mean_degree": lm,
         "thread_max_deg": 8, "warp_max_deg": 256, "block_max_deg": 2048, "coop_blocks_per_sm": 0,
         "vertices_per_block": 2048, "note": "ignored \"quoted\" text", "trials": [1, 2.5, None, True]}
    e.update(shape)
    return e


def _cache(tmp_path, entries, name="cache.json"):
    p = tmp_path / name
    p.write_text(json.dumps({"format": 1, "entries": entries}))
    return str(p)


def test_defaults():
    assert lg.leiden_tuning_default().as_dict() == {"thread_max_deg": 8, "warp_max_deg": 256, "block_max_deg": 2048,
                                                    "coop_blocks_per_sm": 0, "vertices_per_block": 2048,
                                                    "list_order_min_vertices": 1 << 20}


def test_lookup_reads_the_list_order_threshold(tmp_path):
    """An entry may set list_order_min_vertices (0: never); entries without
    it keep the default."""
    path = _cache(tmp_path, [_entry(0, 10, 3, list_order_min_vertices=0)])
    assert lg.leiden_tuning_lookup(path, GPU, 1 << 10, 8 << 10, 10).as_dict()["list_order_min_vertices"] == 0
    path = _cache(tmp_path, [_entry(0, 10, 3)])
    assert lg.leiden_tuning_lookup(path, GPU, 1 << 10, 8 << 10, 10).as_dict()["list_order_min_vertices"] == 1 << 20
    path = _cache(tmp_path, [_entry(0, 10, 3, list_order_min_vertices=-5)])  # outside the range: no entry
    assert lg.leiden_tuning_lookup(path, GPU, 1 << 10, 8 << 10, 10) is None


def test_every_candidate_shape_is_valid(tmp_path):
    """The autotuner searches every field of the launch shape, and each of
    its candidate values passes the library's range checks (a cache entry
    holding it is taken)."""
    assert set(tune.CANDIDATES) == set(lg.leiden_tuning_default().as_dict())
    for key, values in tune.CANDIDATES.items():
        for v in values:
            shape = {key: v}
            if key == "warp_max_deg":
                shape["block_max_deg"] = max(v, 2048)
            path = _cache(tmp_path, [_entry(0, 10, 3, **shape)])
            t = lg.leiden_tuning_lookup(path, GPU, 1 << 10, 8 << 10, 10)
            assert t is not None and t.as_dict()[key] == v, (key, v)


def test_lookup_takes_the_nearest_entry_of_the_same_gpu_and_tail(tmp_path):
    path = _cache(tmp_path, [
        _entry(0, 22, 2, vertices_per_block=1024),          # light, 4M vertices, mean degree 4
        _entry(0, 14, 4, warp_max_deg=128),                 # light, 16k vertices, mean degree 16
        _entry(1, 21, 7, block_max_deg=1024),               # heavy-tailed
        dict(_entry(0, 25, 2, thread_max_deg=4), gpu="another GPU"),
    ])
    # a road-like graph (25M vertices, mean degree 3.6): the light 2^22 entry
    t = lg.leiden_tuning_lookup(path, GPU, 25_000_000, 91_000_000, 8)
    assert t.as_dict()["vertices_per_block"] == 1024 and t.as_dict()["thread_max_deg"] == 8
    # a small block model: the 2^14 entry
    assert lg.leiden_tuning_lookup(path, GPU, 20_000, 300_000, 40).as_dict()["warp_max_deg"] == 128
    # an R-MAT-like graph (largest degree far above 64 times the mean): the heavy entry
    assert lg.leiden_tuning_lookup(path, GPU, 1 << 25, 3_554_875_526, 1_554_551).as_dict()["block_max_deg"] == 1024
    # another GPU's entries are not taken
    assert lg.leiden_tuning_lookup(path, "NVIDIA B200", 1 << 25, 1 << 26, 4) is None
    # the other GPU name selects its own entry
    assert lg.leiden_tuning_lookup(path, "another GPU", 1 << 25, 1 << 26, 4).as_dict()["thread_max_deg"] == 4


def test_lookup_ties_go_to_the_first_entry(tmp_path):
    path = _cache(tmp_path, [_entry(0, 10, 3, vertices_per_block=4096), _entry(0, 12, 3, vertices_per_block=1024)])
    assert lg.leiden_tuning_lookup(path, GPU, 1 << 11, 8 << 11, 10).as_dict()["vertices_per_block"] == 4096


def test_lookup_rejects_bad_caches(tmp_path):
    assert lg.leiden_tuning_lookup(str(tmp_path / "missing.json"), GPU, 10, 10, 2) is None
    bad = tmp_path / "bad.json"
    bad.write_text('{"format": 1, "entries": [ {"gpu": "NVIDIA GB300", ')
    assert lg.leiden_tuning_lookup(str(bad), GPU, 10, 10, 2) is None
    assert "JSON" in lg.leiden_last_error()
    out_of_range = _cache(tmp_path, [_entry(0, 3, 1, warp_max_deg=512)], "range.json")
    assert lg.leiden_tuning_lookup(out_of_range, GPU, 10, 20, 2) is None
    assert "range" in lg.leiden_last_error()
    no_entries = tmp_path / "none.json"
    no_entries.write_text('{"format": 1}')
    assert lg.leiden_tuning_lookup(str(no_entries), GPU, 10, 20, 2) is None


@pytest.mark.parametrize("n,nnz,maxdeg", [(25_000_000, 90_981_444, 8), (1 << 25, 3_554_875_526, 1_554_551),
                                          (10_000, 149_260, 32), (200, 398, 199), (1, 0, 0)])
def test_python_class_matches_the_library(tmp_path, n, nnz, maxdeg):
    """tune.graph_class (what the tuner writes) and the library's lookup
    classify a graph alike: a cache holding only that class's entry and one
    far away always returns the former."""
    c = tune.graph_class(n, nnz, maxdeg)
    far = _entry(1 - c["heavy_tailed"], c["log2_vertices"], c["log2_mean_degree"], vertices_per_block=4096)
    near = _entry(c["heavy_tailed"], c["log2_vertices"], c["log2_mean_degree"], vertices_per_block=1024)
    path = _cache(tmp_path, [far, near])
    assert lg.leiden_tuning_lookup(path, GPU, n, nnz, maxdeg).as_dict()["vertices_per_block"] == 1024
    assert c["heavy_tailed"] == int(maxdeg * n > 64 * nnz)
    if n > 1:
        assert c["log2_vertices"] == round(math.log2(n))


def test_merge_cache_replaces_the_same_class(tmp_path):
    path = str(tmp_path / "c.json")
    tune.merge_cache(path, [_entry(0, 10, 3, vertices_per_block=1024), _entry(1, 10, 3)])
    cache = tune.merge_cache(path, [_entry(0, 10, 3, vertices_per_block=4096)])
    light = [e for e in cache["entries"] if e["heavy_tailed"] == 0]
    assert len(cache["entries"]) == 2 and len(light) == 1 and light[0]["vertices_per_block"] == 4096


_FUZZ = r'''
import json, random, sys
import paper_2312_13936_gb300 as lg
path, out = sys.argv[1], sys.argv[2]
base = open(lg.TUNING_CACHE).read()
rng = random.Random(7)
special = '{}[]",:0123456789.-+eE \\ntfu'
taken = 0
for k in range(400):
    s = list(base)
    for _ in range(rng.randint(1, 6)):
        if not s:
            break
        i = rng.randrange(len(s))
        op = rng.randrange(4)
        if op == 0:
            del s[i:i + rng.randint(1, 40)]
        elif op == 1:
            s[i:i] = s[i:i + rng.randint(1, 40)]
        elif op == 2:
            s[i] = rng.choice(special)
        else:
            s = s[:i]
    text = ''.join(s) if k % 50 else '[' * 100000 + ']' * 100000
    open(out, 'w').write(text)
    t = lg.leiden_tuning_lookup(out, 'NVIDIA GB300', 25_000_000, 90_981_444, 8)
    if t is not None:
        taken += 1
        d = t.as_dict()
        assert 1 <= d['thread_max_deg'] <= 8 and d['warp_max_deg'] <= d['block_max_deg'], d
print('ok', taken)
'''


def test_lookup_survives_mutated_caches(tmp_path):
    """The cache reader (host C++) on 400 random mutations of the shipped
    cache -- spans deleted, repeated or truncated, bytes replaced by JSON
    punctuation, and nesting 100,000 deep -- returns an entry within the
    valid ranges or refuses the file; it never crashes the process (run in a
    subprocess so a crash fails the test)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fuzz.py"
    script.write_text(_FUZZ)
    r = subprocess.run([sys.executable, str(script), lg.TUNING_CACHE, str(tmp_path / "m.json")], cwd=root,
                       capture_output=True, text=True, timeout=300, env=dict(os.environ, PYTHONPATH=root))
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.returncode, r.stdout[-500:], r.stderr[-2000:])
