"""Flop and memory bookkeeping against the paper's printed worked examples
(tests/golden/paper_worked_examples.json, Sec. 4.8) and listing counts."""
import json
import os

import pytest

from paper_1602_06589_gb300 import flops

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_worked_examples.json")))


@pytest.mark.parametrize("ex", GOLD["memory_backup_GiB"])
def test_paper_memory_examples(ex):
    gib = flops.paper_memory_bytes(ex["N_A"], ex["N_L"], ex["N_G"], backup=True) / 2 ** 30
    assert gib == pytest.approx(ex["GiB"], abs=0.05)  # printed to 2-3 significant digits


def test_paper_memory_inconsistency_is_recorded():
    ex = GOLD["memory_not_reproducible"][0]
    gib = flops.paper_memory_bytes(ex["N_A"], ex["N_L"], ex["N_G"], backup=True) / 2 ** 30
    assert gib == pytest.approx(12.82, abs=0.01) and abs(gib - ex["GiB_printed"]) > 5


@pytest.mark.parametrize("ex", GOLD["large_update_share_percent"])
def test_paper_large_update_share(ex):
    # the listing counts reproduce the printed shares to within 0.25 points
    share = 100 * flops.paper_listing_flops(ex["N_A"], ex["N_L"], ex["N_G"], ex["hpd_fraction"])["share"]
    assert share == pytest.approx(ex["percent"], abs=0.25)


def test_algorithmic_flops_relation_to_listings():
    # triangle-only H = W^H (T W) needs half the large-update flops of the
    # paper's zher2k + zgemm pair for H, and the same as its two zherk for S.
    na, nl, ng = 64, 121, 12000
    a = flops.algorithmic_flops(ng, [nl] * na)
    assert a["depth"] == 2 * na * nl
    s_half = a["F_HS"] / 2
    assert s_half == pytest.approx(8 * na * nl * ng ** 2, rel=2 / ng)
    assert a["F_T"] == 32 * ng * na * nl ** 2
