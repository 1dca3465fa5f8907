"""The launch table shipped with the package (tuned.json, measured on B300) is well
formed: every entry is a candidate the autotuner would try, on a key it builds."""
import json

from paper_2305_07450_b300 import autotune


def test_shipped_table_is_well_formed():
    with open(autotune.SHIPPED) as f:
        table = json.load(f)
    assert table, "empty table"
    fwd = {(bx, by) for bx, by in autotune.FWD_CANDIDATES}
    bat = {(bx, by) for bx, by in autotune.BATCH_CANDIDATES}
    n_fwd = 0
    for key, entry in table.items():
        kind = key.split("|")[0]
        launch = entry["launch"]
        assert entry["ms"] > 0 and entry["candidates"]
        assert min(entry["candidates"].values()) == round(entry["ms"], 4) or entry["ms"] <= min(
            entry["candidates"].values()) + 1e-4
        if kind == "fwd":
            n_fwd += 1
            assert len(key.split("|")) == 11
            assert (launch["block_x"], launch["block_y"]) in fwd and launch["staging"] in (1, 2)
        else:
            assert kind == "batch" and (launch["block_x"], launch["block_y"]) in bat
    assert n_fwd >= 8
