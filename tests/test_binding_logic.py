"""Host-side decisions of the Python binding (no GPU needed)."""
import pytest


def test_flag_budget_decision(monkeypatch):
    import paper_2011_11134_gb300 as dg

    monkeypatch.delenv("DGAL_FLAG_BUDGET_BYTES", raising=False)
    assert dg.flag_budget_bytes() == dg.DEFAULT_FLAG_BUDGET_BYTES == 64 << 20
    # 10^7 quadrilateral pairs keep 90 MB of flags: above the default budget
    assert dg.choose_recompute(10_000_000, 4) is True
    assert dg.choose_recompute(1_000_000, 4) is False
    # K = 8 takes 17 bytes a pair
    assert dg.choose_recompute(4_000_000, 8) is True and dg.choose_recompute(3_000_000, 8) is False
    # the boundary is inclusive, an explicit mode wins, the environment sets the default
    assert dg.choose_recompute(100, 4, budget=900) is False and dg.choose_recompute(100, 4, budget=899) is True
    assert dg.choose_recompute(10_000_000, 4, recompute=False) is False
    assert dg.choose_recompute(1, 4, recompute=True) is True
    monkeypatch.setenv("DGAL_FLAG_BUDGET_BYTES", "8")
    assert dg.choose_recompute(1, 4) is True and dg.choose_recompute(1, 4, budget=9) is False
