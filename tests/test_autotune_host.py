"""Host logic of the kernel-variant autotuner: candidates per grid, the
choice of the fastest measured variant, and the JSON cache (a stored choice
is reused without measuring; another grid or precision is measured)."""
import json

from paper_2304_01125_gb300 import autotune as A


def test_candidates_follow_the_fused_pass_support():
    assert A.candidates((64, 64, 64)) == [0, 2, 1, 3]
    assert A.candidates((48, 48, 48)) == [0, 2]      # n0 not a power of two
    assert A.candidates((64, 1, 1)) == [0, 2]        # a line: no 2-D transforms
    assert A.candidates((256, 256, 1)) == [0, 2, 1, 3]


def test_best_variant_measures_once_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def fake(n, prec, v):
        calls.append((n, prec, v))
        return {0: 1.0, 1: 0.7, 2: 1.2, 3: 0.9}[v]

    assert A.best_variant((64, 64, 64), "mixed", "GPU", path=path, measure_fn=fake) == 1
    assert len(calls) == 4
    d = json.load(open(path))
    e = d["GPU|64x64x64|mixed"]
    assert e["kernel_variant"] == 1 and set(e["ms_per_gmres_iteration"]) == {"0", "1", "2", "3"}
    # cached: no measurement
    assert A.best_variant((64, 64, 64), "mixed", "GPU", path=path, measure_fn=fake) == 1
    assert len(calls) == 4
    # another precision and a grid without the fused pass are measured
    assert A.best_variant((64, 64, 64), "fp64", "GPU", path=path, measure_fn=fake) == 1
    assert A.best_variant((48, 48, 48), "mixed", "GPU", path=path, measure_fn=fake) == 0
    assert len(calls) == 4 + 4 + 2
    assert set(json.load(open(path))) == {"GPU|64x64x64|mixed", "GPU|64x64x64|fp64",
                                          "GPU|48x48x48|mixed"}
    # refresh re-measures
    A.best_variant((64, 64, 64), "mixed", "GPU", path=path, measure_fn=fake, refresh=True)
    assert len(calls) == 14


def test_unfused_choice_is_cached_apart(tmp_path):
    path = str(tmp_path / "c.json")
    seen = []

    def fake(n, prec, v):
        seen.append(v)
        return {0: 1.0, 1: 0.5, 2: 0.9, 3: 0.6}[v]

    assert A.best_variant((64, 64, 64), "mixed", "GPU", path=path, measure_fn=fake) == 1
    assert A.best_variant((64, 64, 64), "mixed", "GPU", path=path, measure_fn=fake,
                          fused=False) == 2
    assert sorted(seen) == [0, 0, 1, 2, 2, 3]
    assert A.candidates((64, 64, 64), fused=False) == [0, 2]


def test_damaged_cache_entries_are_measured_again(tmp_path):
    """A malformed file, an entry without a variant, a variant the grid
    cannot run (the fused pass on 48^3) or a non-integer one: measured
    again and replaced."""
    path = tmp_path / "c.json"
    calls = []

    def fake(n, prec, v):
        calls.append(v)
        return {0: 1.0, 1: 0.5, 2: 0.9, 3: 0.6}[v]

    for bad in ("[1, 2]", "{not json",
                json.dumps({"GPU|48x48x48|mixed": {}}),
                json.dumps({"GPU|48x48x48|mixed": {"kernel_variant": 1}}),
                json.dumps({"GPU|48x48x48|mixed": {"kernel_variant": "2"}}),
                json.dumps({"GPU|48x48x48|mixed": {"kernel_variant": True}})):
        path.write_text(bad)
        calls.clear()
        assert A.best_variant((48, 48, 48), "mixed", "GPU", path=str(path),
                              measure_fn=fake) == 2
        assert sorted(calls) == [0, 2]
        assert json.loads(path.read_text())["GPU|48x48x48|mixed"]["kernel_variant"] == 2


def test_unwritable_cache_still_returns_the_choice(tmp_path):
    """A cache path that cannot be written (its folder is a file): the
    measured choice is returned all the same."""
    blocker = tmp_path / "file"
    blocker.write_text("")
    path = str(blocker / "sub" / "c.json")
    got = A.best_variant((64, 64, 64), "mixed", "GPU", path=path,
                         measure_fn=lambda n, p, v: {0: 1.0, 1: 2.0, 2: 0.5, 3: 3.0}[v])
    assert got == 2
