"""Host logic of the cluster-size cache (no GPU): the key names the device,
each simulation's shape-setting options and the jobs of every level; the
table survives a round trip and a damaged file reads as empty."""
import json
import os
from types import SimpleNamespace

from paper_2512_07615_gb300 import tnlbm as T


def cfg(n=6, lattice=19, chi=64, precision=3, max_cluster=0, sweeps=2):
    return SimpleNamespace(n_per_axis=n, lattice=lattice, chi_max=chi, precision=precision,
                           max_cluster=max_cluster, sweeps=sweeps)


def test_key_names_device_configs_and_jobs():
    k = T.cluster_cache_key("GB300", [cfg(), cfg(chi=32)], [0, 24, 11])
    assert k == T.cluster_cache_key("GB300", [cfg(), cfg(chi=32)], [0, 24, 11])
    others = [T.cluster_cache_key("B200", [cfg(), cfg(chi=32)], [0, 24, 11]),
              T.cluster_cache_key("GB300", [cfg(chi=32), cfg()], [0, 24, 11]),
              T.cluster_cache_key("GB300", [cfg(), cfg(chi=32, precision=0)], [0, 24, 11]),
              T.cluster_cache_key("GB300", [cfg(), cfg(chi=32)], [0, 24, 12]),
              T.cluster_cache_key("GB300", [cfg(), cfg(chi=32, max_cluster=4)], [0, 24, 11])]
    assert len(set(others + [k])) == len(others) + 1
    d = json.loads(k)
    assert d["device"] == "GB300" and d["jobs"] == [0, 24, 11] and d["sims"][1][2] == 32


def test_store_and_load_round_trip(tmp_path):
    path = str(tmp_path / "clusters.json")
    assert T.load_cluster_cache(path) == {}
    T.store_cluster_cache(path, "a", [0, 4, 4])
    T.store_cluster_cache(path, "b", (0, 16, 12))
    T.store_cluster_cache(path, "a", [0, 8, 4])
    assert T.load_cluster_cache(path) == {"a": [0, 8, 4], "b": [0, 16, 12]}
    assert sorted(os.listdir(tmp_path)) == ["clusters.json"]     # no temporary file left


def test_damaged_or_foreign_file_reads_as_empty(tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert T.load_cluster_cache(str(bad)) == {}
    lst = tmp_path / "list.json"
    lst.write_text("[1, 2, 3]")
    assert T.load_cluster_cache(str(lst)) == {}
    T.store_cluster_cache(str(bad), "k", [1])
    assert T.load_cluster_cache(str(bad)) == {"k": [1]}
