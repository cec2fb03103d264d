"""The launch-parameter table (rips_set_tuning / rips_get_tuning): host-side
behaviour only, no GPU needed."""
import pytest

from paper_1908_02518_gb300 import tuning, _lib


@pytest.fixture(autouse=True)
def _clean_table():
    tuning.clear_tuning()
    yield
    tuning.clear_tuning()


def test_defaults_when_nothing_matches():
    assert tuning.get_tuning(1, 1000) == tuning.DEFAULT
    assert tuning.get_tuning(7, 1) == tuning.DEFAULT


def test_entry_applies_to_its_dimension_and_size_range():
    p = {"warp_chain_limit": 8, "warp_merge_max": 512, "reduce_blocks_per_sm": 1, "scan_blocks_per_sm": 32}
    tuning.set_tuning(2, 513, 1024, p)
    assert tuning.get_tuning(2, 513) == p
    assert tuning.get_tuning(2, 1024) == p
    assert tuning.get_tuning(2, 512) == tuning.DEFAULT
    assert tuning.get_tuning(2, 1025) == tuning.DEFAULT
    assert tuning.get_tuning(1, 600) == tuning.DEFAULT


def test_later_entries_take_precedence_and_clear_forgets():
    tuning.set_tuning(1, 1, 10**6, {"warp_chain_limit": 8})
    tuning.set_tuning(1, 100, 200, {"warp_chain_limit": 128})
    assert tuning.get_tuning(1, 150)["warp_chain_limit"] == 128
    assert tuning.get_tuning(1, 50)["warp_chain_limit"] == 8
    tuning.clear_tuning()
    assert tuning.get_tuning(1, 150) == tuning.DEFAULT


@pytest.mark.parametrize("dim,lo,hi,p", [
    (0, 1, 10, {}), (8, 1, 10, {}), (1, 10, 5, {}), (1, 0, 5, {}),
    (1, 1, 10, {"warp_chain_limit": 0}), (1, 1, 10, {"warp_merge_max": 0}),
    (1, 1, 10, {"reduce_blocks_per_sm": -1}), (1, 1, 10, {"scan_blocks_per_sm": 0}),
    (1, 1, 10, {"scan_blocks_per_sm": 65}),
])
def test_out_of_range_is_rejected(dim, lo, hi, p):
    with pytest.raises(_lib.RipsError):
        tuning.set_tuning(dim, lo, hi, p)


def test_buckets_are_powers_of_two():
    assert tuning.bucket(1) == (1, 1)
    assert tuning.bucket(512) == (257, 512)
    assert tuning.bucket(513) == (513, 1024)
    assert tuning.bucket(1000) == (513, 1024)


def test_save_and_load_round_trip(tmp_path):
    table = {1: {"params": dict(tuning.DEFAULT, warp_chain_limit=8), "ms": 1.0, "default_ms": 2.0,
                 "bucket": [257, 512]}}
    path = str(tmp_path / "t.json")
    tuning.save(table, path)
    tuning.clear_tuning()
    tuning.load(path)
    assert tuning.get_tuning(1, 300)["warp_chain_limit"] == 8


def test_limits_round_trip_and_validation():
    import paper_1908_02518_gb300 as rg
    try:
        rg.set_limits(barrier_wait_ns=5, chain_ns=6, arena_entries=7, table_slots=64)
        assert rg.get_limits() == {"barrier_wait_ns": 5, "chain_ns": 6, "arena_entries": 7, "table_slots": 64}
        for bad in (3, 100, 1 << 40):
            with pytest.raises(_lib.RipsError):
                rg.set_limits(table_slots=bad)
    finally:
        rg.set_limits()
    assert rg.get_limits() == {"barrier_wait_ns": 0, "chain_ns": 0, "arena_entries": 0, "table_slots": 0}
