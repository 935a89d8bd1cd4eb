"""Host logic of the benchmark that needs no GPU: the DRAM traffic of a Dslash
launch is taken from the stored ncu summary only while that summary was
captured on the current kernel sources, and it scales with the number of
output sites; the batched kernel's entries are keyed by right-hand-side
count."""
import json
import os

import bench
from paper_2502_00152_gb300.build import dslash_source_hash


def _write(root, doc):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", "dslash_traffic.json"), "w") as f:
        json.dump(doc, f)


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    per_site = {"oe_s16_r12": 987.6, "mrhs12_oe_s16_r12": 1331.5}
    _write(root, {"kernel_source_hash": dslash_source_hash(), "dram_bytes_per_output_site": per_site})
    assert bench.ncu_traffic("oe_s16_r12", 1000) == 987.6 * 1000
    assert bench.ncu_traffic("mrhs12_oe_s16_r12", 12582912) == 1331.5 * 12582912
    assert bench.ncu_traffic("mrhs24_oe_s16_r12", 1000) is None  # not captured for 24 right-hand sides
    # a summary taken on other kernel sources is not used
    _write(root, {"kernel_source_hash": "0" * 16, "dram_bytes_per_output_site": per_site})
    assert bench.ncu_traffic("oe_s16_r12", 1000) is None
    # nor a missing or unreadable one
    os.remove(os.path.join(root, "profiles", "dslash_traffic.json"))
    assert bench.ncu_traffic("oe_s16_r12", 1000) is None


def test_committed_traffic_names_its_commands():
    """The committed summary says how each figure was made, and its figures are
    close to the algorithmic bytes of the kernels (links read once, each field
    once): no re-reads."""
    with open(os.path.join(bench.ROOT, "profiles", "dslash_traffic.json")) as f:
        d = json.load(f)
    assert d["commands"] and all(c.startswith("ncu ") and "--clock-control none" in c for c in d["commands"])
    algorithmic = {"oe_s16_r12": 960 + 2 * 16, "mrhs12_oe_s16_r12": 960 + 12 * 2 * 16,
                   "mrhs12_eo_s16_r12": 960 + 12 * (16 + 16 + 16 + 16 + 24 + 24)}
    for key, alg in algorithmic.items():
        got = d["dram_bytes_per_output_site"][key]
        assert 0.9 * alg <= got <= 1.1 * alg, (key, got, alg)
