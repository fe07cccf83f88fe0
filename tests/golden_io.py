"""Reader for the hand-worked fixtures in tests/golden/."""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok: str, wtype: int):
    if wtype == 1:
        return int(tok)
    return float(tok)


def load(path: str) -> dict:
    d = dict(edges=[], parent={})
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "n":
            d["n"] = int(tok[1])
        elif tok[0] == "wtype":
            d["wtype"] = 0 if tok[1] == "f32" else 1
        elif tok[0] == "edge":
            d["edges"].append((int(tok[1]), int(tok[2]), tok[3]))
        elif tok[0] == "mask":
            d["mask"] = np.array([int(t) for t in tok[1:]], np.uint8)
        elif tok[0] == "labels":
            d["labels"] = np.array([int(t) for t in tok[1:]], np.int32)
        elif tok[0] == "total":
            d["total"] = float(tok[1])
        elif tok[0] == "rounds":
            d["rounds"] = int(tok[1])
        elif tok[0] == "parent":
            d["parent"][int(tok[1])] = np.array([int(t) for t in tok[2:]], np.int64)
    wt = d["wtype"]
    d["src"] = np.array([e[0] for e in d["edges"]], np.int32)
    d["dst"] = np.array([e[1] for e in d["edges"]], np.int32)
    if wt == 0:
        d["w"] = np.array([float(e[2]) for e in d["edges"]], np.float32)
    else:
        d["w"] = np.array([int(e[2]) for e in d["edges"]], np.uint32)
    d["name"] = os.path.basename(path)
    return d


def all_fixtures():
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]


def load_connectivity(path: str) -> dict:
    """A hand-worked connectivity fixture (tests/golden/connectivity/): edges,
    the round count, the labels, and per round k the parents after
    conditional hooking (cond k), the star flags after it (star k), the
    parents after unconditional hooking (uncond k) and after shortcutting
    (parent k)."""
    d = dict(edges=[], cond={}, star={}, uncond={}, parent={})
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "n":
            d["n"] = int(tok[1])
        elif tok[0] == "edge":
            d["edges"].append((int(tok[1]), int(tok[2])))
        elif tok[0] == "rounds":
            d["rounds"] = int(tok[1])
        elif tok[0] == "labels":
            d["labels"] = np.array([int(t) for t in tok[1:]], np.int32)
        elif tok[0] in ("cond", "star", "uncond", "parent"):
            d[tok[0]][int(tok[1])] = np.array([int(t) for t in tok[2:]], np.int64)
    d["src"] = np.array([e[0] for e in d["edges"]], np.int32)
    d["dst"] = np.array([e[1] for e in d["edges"]], np.int32)
    d["name"] = os.path.basename(path)
    return d


def connectivity_fixtures():
    return [load_connectivity(p)
            for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "connectivity", "*.txt")))]
