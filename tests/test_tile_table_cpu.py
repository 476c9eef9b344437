"""The tile table's host logic (CPU only): the library's JSON reader, rule
validation and the selection of a rule for (precision, N), plus the shape of
the tuned table shipped with the package.  No device is touched."""
import json
import os

import pytest

from paper_1204_3052_gb300 import matpow as mpw

TABLE = {
    "version": 1,
    "device": "NVIDIA GB300",
    "note": "ignored keys may hold anything: [1, {\"x\": null}]",
    "rules": [
        {"precision": "bf16x6", "n_lo": 64, "n_hi": 128, "bn": 64, "split_k": 2, "chain": 1,
         "persist": 1, "us": 12.5, "candidates": [{"bn": 64, "us": 13.0}]},
        {"precision": "bf16x3", "n_lo": 1024, "n_hi": 8192, "bn": 128},
        {"precision": 2, "n_lo": 2048, "n_hi": 4096, "bn": 64, "persist": 0},
        {"precision": "fp32", "n_lo": 0, "n_hi": 64, "chain": None},
    ],
}


def test_parse_reads_every_field_and_skips_the_rest():
    st, rules = mpw.matpow_tile_table_parse(json.dumps(TABLE))
    assert st == mpw.OK and len(rules) == 4
    assert rules[0] == {"n_lo": 64, "n_hi": 128, "precision": mpw.BF16X6, "bn": 64, "split_k": 2,
                        "chain": 1, "persist": 1}
    # omitted fields and null are -1 (the built-in choice)
    assert rules[1] == {"n_lo": 1024, "n_hi": 8192, "precision": mpw.BF16X3, "bn": 128, "split_k": -1,
                        "chain": -1, "persist": -1}
    assert rules[2]["precision"] == mpw.BF16X3 and rules[2]["persist"] == 0
    assert rules[3]["chain"] == -1 and rules[3]["precision"] == mpw.FP32_SIMT


def test_parse_rejects_malformed_text_with_a_position():
    lib = mpw.load()
    for bad in ('{"rules": [ {"bn": 64,} ]}', '{"rules": [}', '[1, 2]', '{"rules": 3}',
                '{"rules": [{"precision": "fp16"}]}', '{"rules": [{"bn": 6.5}]}',
                '{"x": 1}', '{"rules": []} extra', '{"rules": [{"bn": 64}'):
        st, _ = mpw.matpow_tile_table_parse(bad)
        assert st == mpw.EINVAL, bad
        msg = lib.matpow_last_error(None).decode()
        assert "tile table" in msg, (bad, msg)
    st, rules = mpw.matpow_tile_table_parse('  {"rules": []}\n')
    assert st == mpw.OK and rules == []


def test_lookup_takes_the_last_covering_rule_of_the_precision():
    _, rules = mpw.matpow_tile_table_parse(json.dumps(TABLE))
    # (64, 128] for bf16x6: N = 64 is outside, 65 and 128 inside
    assert mpw.matpow_tile_rule_lookup(rules, "bf16x6", 64)[0] == mpw.EAGAIN
    for N in (65, 100, 128):
        st, r = mpw.matpow_tile_rule_lookup(rules, "bf16x6", N)
        assert st == mpw.OK and r["split_k"] == 2, N
    assert mpw.matpow_tile_rule_lookup(rules, "bf16x6", 129)[0] == mpw.EAGAIN
    # bf16x3: (1024, 8192] then (2048, 4096] later in the table wins where both cover
    assert mpw.matpow_tile_rule_lookup(rules, "bf16x3", 1500)[1]["bn"] == 128
    st, r = mpw.matpow_tile_rule_lookup(rules, "bf16x3", 3000)
    assert st == mpw.OK and r["bn"] == 64 and r["persist"] == 0
    assert mpw.matpow_tile_rule_lookup(rules, "bf16x3", 5000)[1]["bn"] == 128
    # another precision never matches
    st, r = mpw.matpow_tile_rule_lookup(rules, "bf16", 3000)
    assert st == mpw.EAGAIN and r["bn"] == -1 and r["precision"] == mpw.BF16


def test_set_table_validates_rules():
    lib = mpw.load()
    good = mpw._rules_array([{"precision": "bf16x6", "n_lo": 64, "n_hi": 128, "bn": 64}])
    # no plan on this machine: a NULL plan is refused before the rules are read
    assert lib.matpow_plan_set_tile_table(None, good, 1) == mpw.EINVAL
    assert lib.matpow_plan_load_tile_table(None, b"/nonexistent") == mpw.EINVAL


@pytest.mark.skipif(not os.path.exists(mpw.DEFAULT_TILE_TABLE), reason="no tuned table shipped")
def test_shipped_table_parses_and_is_well_formed():
    text = open(mpw.DEFAULT_TILE_TABLE).read()
    st, rules = mpw.matpow_tile_table_parse(text)
    assert st == mpw.OK and rules
    for r in rules:
        assert 0 <= r["n_lo"] < r["n_hi"]
        assert r["bn"] in (-1, 64, 128) and r["split_k"] in (-1, 1, 2, 4)
        assert r["chain"] in (-1, 0, 1) and r["persist"] in (-1, 0, 1)
        if r["precision"] == mpw.BF16X6:
            assert r["bn"] in (-1, 64)  # three accumulators per buffer fit TMEM at 64 columns
    meta = json.loads(text)
    assert meta.get("device") and meta.get("measured")
