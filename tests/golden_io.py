"""Reader for the hand-derived fixtures in tests/golden/ (format documented in each file)."""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


class Golden:
    def __init__(self, path):
        self.path = path
        self.name = os.path.basename(path)
        self.nets, self.gains, self.rounds = [], [], []
        self.vertex_w = self.net_w = None
        self.final = None
        for line in open(path):
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "net":
                self.nets.append([int(v) for v in vals])
            elif key == "gain":
                self.gains.append(tuple(int(v) for v in vals))
            elif key == "round":
                self.rounds.append(tuple(int(v) for v in vals))
            elif key == "part":
                self.part = np.array([int(v) for v in vals], dtype=np.int32)
            elif key == "final":
                self.final = np.array([int(v) for v in vals], dtype=np.int32)
            elif key == "vertex_weights":
                self.vertex_w = np.array([int(v) for v in vals], dtype=np.int32)
            elif key == "net_weights":
                self.net_w = np.array([int(v) for v in vals], dtype=np.int32)
            elif key == "eps":
                self.eps = float(vals[0])
            else:
                setattr(self, key, int(vals[0]))
        self.m = len(self.nets)
        self.net_off = np.zeros(self.m + 1, dtype=np.int64)
        self.net_off[1:] = np.cumsum([len(e) for e in self.nets])
        self.pins = np.array([v for e in self.nets for v in e], dtype=np.int32)


def load_all():
    return [Golden(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
