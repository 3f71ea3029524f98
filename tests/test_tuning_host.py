"""Host logic of the autotuning cache: size classes and the JSON round trip."""
import json

from paper_2509_26279_gb300 import tuning
from paper_2509_26279_gb300 import workloads as W


def test_size_classes_group_similar_fields():
    g = W.decam_tno().grid
    a = tuning.size_class(100, 300_000, g, 25)
    assert a == tuning.size_class(110, 330_000, g, 28)      # same epoch step, density, threshold share
    assert a != tuning.size_class(140, 300_000, g, 35)      # other epoch step
    assert a != tuning.size_class(100, 1_200_000, g, 25)    # 4x the density
    assert a != tuning.size_class(100, 300_000, W.fast_movers().grid, 25)


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    c = tuning.TuneCache(p)
    c.entries["E4-d11-v111x111-b2000-f2"] = {"superbin": 3, "velocity_block": 4, "ms": 2.5, "device": "x"}
    c.save()
    c2 = tuning.TuneCache(p)
    assert c2.lookup("E4-d11-v111x111-b2000-f2")["superbin"] == 3
    assert json.load(open(p)) == c.entries


def test_tagged_entries_are_kept_apart():
    """Entries tuned for another search form live under their own key prefix."""
    from paper_2509_26279_gb300 import workloads as W

    class F:
        pass

    w = W.batched_fields(1)[0]
    f = F()
    f.E, f.w = w.recipe.n_epochs, w
    f.cat = W.load(w)
    c = tuning.TuneCache()
    key = tuning.size_class(f.E, f.cat.n, w.grid, w.n_min)
    c.entries[key] = {"tile_kx": 8, "tile_ky": 8, "superbin": 3, "tile_bx": 0, "tile_by": 0, "velocity_block": 0}
    c.entries["peaks_only_e6:" + key] = {"tile_kx": 8, "tile_ky": 4, "superbin": 4, "tile_bx": 64, "tile_by": 0,
                                         "velocity_block": 2}
    assert c.lookup(key)["superbin"] == 3
    assert c.lookup("peaks_only_e6:" + key)["superbin"] == 4
