"""The lane schedule of the persistent row kernel's trailing update.

Panel p of the blocked Cholesky of a g x g tile matrix leaves the trailing
tiles (I, J), p < J <= I < g, each updated as two half-tile units (h = 0, 1).
The schedule in ws_units.inc hands these units to the 32 lanes of a consumer
warp round by round; a unit missing from it would leave a tile un-updated and
a unit listed twice would subtract L_Ip L_Jp^T twice.  So every unit of every
panel must appear exactly once, in the fewest rounds of 32 lanes, and the
bank-group model the schedule was built against must show it costing fewer
shared-memory passes than the plain lane-order assignment it replaced.
"""
import importlib.util
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_04159_gb300", "csrc")


def _table():
    txt = open(os.path.join(CSRC, "ws_units.inc")).read()
    gmin = int(re.search(r"kWsUnitGMin = (\d+)", txt).group(1))
    gmax = int(re.search(r"kWsUnitGMax = (\d+)", txt).group(1))
    body = re.search(r"kWsUnits\[(\d+)\] = \{(.*?)\};", txt, re.S)
    units = [int(v, 16) for v in re.findall(r"0x[0-9a-f]+", body.group(2))]
    assert len(units) == int(body.group(1))
    rb = re.search(r"kWsUnitRound\[(\d+)\]\[(\d+)\] = \{(.*?)\};", txt, re.S)
    rows = [[int(v) for v in r.split(",") if v.strip()] for r in re.findall(r"\{([^{}]*)\}", rb.group(3))]
    assert len(rows) == gmax - gmin + 1
    return gmin, gmax, units, rows


def _gen():
    spec = importlib.util.spec_from_file_location("gen_ws_units", os.path.join(CSRC, "gen_ws_units.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_unit_once_in_the_fewest_rounds():
    gmin, gmax, units, rows = _table()
    assert gmin <= 2 and gmax >= 16  # K = 8 .. 127
    for g in range(gmin, gmax + 1):
        rnd = rows[g - gmin]
        assert all(b >= a for a, b in zip(rnd, rnd[1:]))
        for p in range(g):
            want = {(I, J, h) for I in range(p + 1, g) for J in range(p + 1, I + 1) for h in (0, 1)}
            got = []
            for e in units[32 * rnd[p]:32 * rnd[p + 1]]:
                if e == 0xFFFF:
                    continue
                assert e >> 9 == 0, hex(e)
                got.append((e & 15, (e >> 4) & 15, (e >> 8) & 1))
            assert len(got) == len(want) and set(got) == want, (g, p)
            assert rnd[p + 1] - rnd[p] == math.ceil(len(want) / 32), (g, p)


def _passes(gen, g, lane_units):
    tot = 0
    for p, lanes in enumerate(lane_units):
        for k in range(0, len(lanes), 8):
            tot += gen.group_cost([u for u in lanes[k:k + 8] if u is not None], p)
    return tot


@pytest.mark.parametrize("g", [5, 13])
def test_schedule_beats_lane_order_under_the_bank_model(g):
    gen = _gen()
    gmin, _, units, rows = _table()
    rnd = rows[g - gmin]
    sched, plain = [], []
    for p in range(g):
        sched.append([None if e == 0xFFFF else (e & 15, (e >> 4) & 15, (e >> 8) & 1)
                      for e in units[32 * rnd[p]:32 * rnd[p + 1]]])
        # the assignment by lane order: unit u = 2 t + h, t the trailing tiles row by row
        plain.append([(I, J, h) for I in range(p + 1, g) for J in range(p + 1, I + 1) for h in (0, 1)])
    s, q = _passes(gen, g, sched), _passes(gen, g, plain)
    assert s < q, (s, q)
    if g == 13:  # K = 100
        assert s <= 0.7 * q, (s, q)


def test_bank_model_special_cases():
    gen = _gen()
    # eight lanes on eight consecutive 16-byte words: one pass
    assert gen.passes([4 * i for i in range(8)]) == 1
    # the same word eight times: a broadcast, one pass
    assert gen.passes([36] * 8) == 1
    # two words 32 floats apart share a bank group: two passes
    assert gen.passes([0, 32]) == 2
    assert gen.passes([0, 32, 64, 4]) == 3


def test_table_is_what_the_seeded_generator_writes():
    """The committed table is reproducible: gen_ws_units.py draws every grid
    from one seeded random stream in order of g, so rerunning it for the
    smallest grids (g <= 8, a prefix of that stream) must give the first
    entries of the table and their round offsets exactly."""
    import random
    gmin, _, units, rows = _table()
    gen = _gen()
    rng = random.Random(gen.SEED)
    flat = []
    for g in range(gen.G_MIN, 9):
        starts = []
        for p in range(g):
            starts.append(len(flat) // 32)
            lanes, _ = gen.schedule(g, p, rng) if p < g - 1 else ([], 0)
            flat += lanes
        starts.append(len(flat) // 32)
        assert starts == rows[g - gmin][:g + 1], g
    assert flat == units[:len(flat)]
