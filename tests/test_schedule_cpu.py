"""The rules that cut a batch into the units of a step schedule (schedule.h),
compiled on the CPU and checked on random batches.

A unit is a range of one group's members.  For every batch, cap and k:
- the units of one group tile its members exactly once, in order;
- a group is cut only when its passes can be sliced, into
  min(members, ceil(points / cap)) ranges (one range with cap 0), whose sizes
  differ by at most one member;
- cutting each unit k ways (the streamed step) again tiles it exactly, into
  min(k, its members) ranges of sizes that differ by at most one.
"""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_19840_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "schedule_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def run(exe, cases):
    text = ""
    for G, cap, k, groups in cases:
        text += f"{G} {cap} {k}\n" + "".join(f"{p} {m} {s}\n" for p, m, s in groups)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    res, cur, lists = [], [], []
    for ln in out:
        if not ln:
            continue
        if ln == "end":
            lists.append(cur)
            cur = []
            if len(lists) == 2:
                res.append(tuple(lists))
                lists = []
            continue
        cur.append(tuple(int(v) for v in ln.split()))
    return res


def tiles(units, group, m0, m1):
    got = [(a, b) for g, a, b in units if g == group]
    assert got and got[0][0] == m0 and got[-1][1] == m1, (got, m0, m1)
    assert all(got[i][1] == got[i + 1][0] for i in range(len(got) - 1)), got
    assert all(b > a for a, b in got), got
    sizes = [b - a for a, b in got]
    assert max(sizes) - min(sizes) <= 1, sizes
    return len(got)


def test_units_tile_every_group_and_respect_the_cap(driver):
    rng = random.Random(7)
    cases = []
    for _ in range(400):
        G = rng.randint(1, 5)
        groups = []
        for _ in range(G):
            m = rng.randint(1, 96)
            npts = rng.choice([256, 1024, 4096, 65536, 262144])
            groups.append((m * npts, m, rng.random() < 0.8))
        total = sum(p for p, _, _ in groups)
        biggest = max(p // m for p, m, _ in groups)
        B = rng.choice([0, 1, 2, 3, 4, 6])
        cap = 0 if B == 0 else max(biggest, -(-total // B))
        cases.append((G, cap, rng.randint(1, 6), [(p, m, int(s)) for p, m, s in groups]))
    for (G, cap, k, groups), (units, split) in zip(cases, run(driver, cases)):
        assert sorted({u[0] for u in units}) == list(range(G))
        for g, (p, m, s) in enumerate(groups):
            want = 1 if (cap == 0 or not s) else min(m, -(-p // cap))
            assert tiles(units, g, 0, m) == want, (groups, cap)
        # cut k ways: every unit tiled by min(k, its members) ranges
        for g, a, b in units:
            inner = [(gg, x, y) for gg, x, y in split if gg == g and a <= x and y <= b]
            assert tiles(inner, g, a, b) == min(k, b - a)
        assert len(split) == sum(min(k, b - a) for _, a, b in units)


def test_known_batches(driver):
    # 64 x 256^2 and 32 x 512^2 (the crossing-sea batch): total/3 keeps the
    # 256^2 group whole and halves the 512^2 group; the streamed step's k = 4
    # makes 12 units
    small, big = 64 * 65536, 32 * 262144
    total = small + big
    cap3 = max(262144, -(-total // 3))
    (units, split), = run(driver, [(2, cap3, 4, [(small, 64, 1), (big, 32, 1)])])
    assert units == [(0, 0, 64), (1, 0, 16), (1, 16, 32)]
    assert len(split) == 12 and split[:4] == [(0, 0, 16), (0, 16, 32), (0, 32, 48), (0, 48, 64)]
    # a group whose passes cannot be sliced stays whole; one member stays one unit
    (units, split), = run(driver, [(2, 1000, 3, [(8192, 4, 0), (4096, 1, 1)])])
    assert units == [(0, 0, 4), (1, 0, 1)] and split == [(0, 0, 1), (0, 1, 2), (0, 2, 4), (1, 0, 1)]
