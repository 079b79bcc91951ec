"""The autotuner's table on the host: text round trip, merge, clear and
rejection of malformed input (no GPU needed: the table lives in the library)."""
import pytest

import paper_2609_02394_b300 as P


@pytest.fixture(autouse=True)
def empty_table():
    P.tune_clear()
    yield
    P.tune_clear()


def test_round_trip_and_merge():
    assert P.tune_dump() == ""
    text = "gram|df|96x96|4096=4\ncomb|f32|t|96x96|4096=1\n"
    assert P.tune_load(text) == 2
    assert P.tune_dump() == "comb|f32|t|96x96|4096=1\ngram|df|96x96|4096=4\n"
    # a later load overrides the same key and keeps the others
    assert P.tune_load("gram|df|96x96|4096=7") == 1
    assert P.tune_dump() == "comb|f32|t|96x96|4096=1\ngram|df|96x96|4096=7\n"
    P.tune_clear()
    assert P.tune_dump() == ""


@pytest.mark.parametrize("bad", ["no equals sign", "=3", "key=", "key=x", "key=-1", "key=3junk"])
def test_malformed_lines_are_rejected(bad):
    with pytest.raises(ValueError):
        P.tune_load(bad)
