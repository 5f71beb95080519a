"""Pins for `oracle.dcsc_tiles`, the 2D blocks of Sec. 3.2 in the DCSC form of Sec. 4.1.

- Fig. 3's matrix split rowwise into two three-row pieces gives the hand-derived
  IR / JC / CP arrays of `tests/golden/fig3_dcsc.json`.
- On random graphs and block sizes it equals a naive builder that walks every
  block with dictionaries (no sorting, no vector arithmetic).
- Reassembling the blocks gives back exactly the entries of the CSR.
- A planted mistake (rows not local to their block) is caught by the golden.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1104_4518_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def csr_of_rows(rows):
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    adj = np.array([u for r in rows for u in r], dtype=np.int32)
    return oracle.CSR(off, adj)


def naive_dcsc(g, R, C):
    n = g.n
    nrb, ncb = (n + R - 1) // R, (n + C - 1) // C
    tdir_jc, tdir_ir, jc, cp, ir = [0], [0], [], [], []
    for rb in range(nrb):
        for cb in range(ncb):
            cols = {}
            for v in range(rb * R, min(n, (rb + 1) * R)):
                for u in g.row(v):
                    if cb * C <= u < (cb + 1) * C:
                        cols.setdefault(int(u) - cb * C, []).append(v - rb * R)
            start = len(ir)
            for c in sorted(cols):
                jc.append(c)
                cp.append(len(ir) - start)
                ir.extend(sorted(cols[c]))
            tdir_jc.append(len(jc))
            tdir_ir.append(len(ir))
    return {"tdir_jc": tdir_jc, "tdir_ir": tdir_ir, "jc": jc, "cp": cp, "ir": ir}


def test_fig3_pieces_match_the_hand_derived_dcsc():
    gold = json.load(open(os.path.join(HERE, "golden", "fig3_dcsc.json")))
    g = csr_of_rows(gold["rows"])
    t = oracle.dcsc_tiles(g, gold["rows_per_piece"], 6)
    assert t["nrb"] == 2 and t["ncb"] == 1
    for k, piece in enumerate(gold["pieces"]):
        j0, j1 = t["tdir_jc"][k], t["tdir_jc"][k + 1]
        i0, i1 = t["tdir_ir"][k], t["tdir_ir"][k + 1]
        assert t["jc"][j0:j1].tolist() == piece["JC"]
        assert t["cp"][j0:j1].tolist() == piece["CP"]
        assert t["ir"][i0:i1].tolist() == piece["IR"]


def test_fig3_golden_catches_global_row_ids():
    gold = json.load(open(os.path.join(HERE, "golden", "fig3_dcsc.json")))
    t = oracle.dcsc_tiles(csr_of_rows(gold["rows"]), gold["rows_per_piece"], 6)
    i0, i1 = t["tdir_ir"][1], t["tdir_ir"][2]
    planted = (t["ir"][i0:i1] + 3).tolist()  # row ids left global: a plausible slip
    assert planted != gold["pieces"][1]["IR"]


@pytest.mark.parametrize("R,C,seed", [(1, 1, 0), (3, 5, 1), (8, 8, 2), (16, 4, 3), (64, 64, 4), (7, 200, 5)])
def test_equals_the_naive_builder(R, C, seed):
    el = inputs.rmat(7, 8, seed=seed)
    g = oracle.csr_of(el)
    got = oracle.dcsc_tiles(g, R, C)
    ref = naive_dcsc(g, R, C)
    for key in ("tdir_jc", "tdir_ir", "jc", "cp", "ir"):
        assert got[key].tolist() == ref[key], key


def test_blocks_reassemble_into_the_csr():
    el = inputs.rmat(10, 16, seed=9)
    g = oracle.csr_of(el)
    R, C = 32, 128
    t = oracle.dcsc_tiles(g, R, C)
    got = set()
    for tile in range(t["ntiles"]):
        rb, cb = divmod(tile, t["ncb"])
        i1 = t["tdir_ir"][tile + 1]
        j0, j1 = t["tdir_jc"][tile], t["tdir_jc"][tile + 1]
        base = t["tdir_ir"][tile]
        for j in range(j0, j1):
            end = base + t["cp"][j + 1] if j + 1 < j1 else i1
            rows = t["ir"][base + t["cp"][j]:end]
            assert np.all(np.diff(rows) > 0)
            for r in rows:
                got.add((rb * R + int(r), cb * C + int(t["jc"][j])))
        assert np.all(np.diff(t["jc"][j0:j1]) > 0)
    want = {(v, int(u)) for v in range(g.n) for u in g.row(v)}
    assert got == want
