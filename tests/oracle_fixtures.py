"""Helpers shared by the oracle tests (parsing of the golden files)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LETTER = {"F": 0, "B": 1, "G": 2, "I": 3}


def read_geometry(name):
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name))]
    lines = [ln for ln in lines if ln and not ln.startswith("#")]
    sec, mask, cls, links = None, [], [], {}
    for ln in lines:
        if ln in ("MASK", "CLASS", "LINKS"):
            sec = ln
            continue
        if sec == "MASK":
            mask.append([int(c) for c in ln])
        elif sec == "CLASS":
            cls.append([LETTER[c] for c in ln])
        elif sec == "LINKS":
            key, *rest = ln.split()
            if key == "node":
                links["node"] = (int(rest[0]), int(rest[1]))
            else:
                links[key] = {tuple(int(v) for v in r.split(",")) for r in rest}
    mask = np.array(mask[::-1], np.uint8)   # file lists the top row first
    cls = np.array(cls[::-1], np.uint8)
    return mask, cls, links


def read_lattice():
    rows = []
    for ln in open(os.path.join(GOLDEN, "d2q9_paper_order.txt")):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            rows.append([int(v) for v in ln.split()])
    a = np.array(rows)
    return a[:, 1], a[:, 2], a[:, 3] / a[:, 4]
