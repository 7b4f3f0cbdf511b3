"""Reader for the hand-worked examples under tests/golden/."""
from __future__ import annotations

import glob
import math
import os
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Golden:
    name: str
    metric: str
    x: np.ndarray
    a: np.ndarray
    y: np.ndarray
    b: np.ndarray
    nn: dict = field(default_factory=dict)     # round -> list of supplier ids
    plan: list = field(default_factory=list)   # (i, j, f)
    rounds: int = 0
    cost: float = 0.0
    cost_expr: str = ""
    emd: float = 0.0

    def cost_from_expr(self) -> float:
        return float(eval(self.cost_expr, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def load(path: str) -> Golden:
    metric = None
    S, C = [], []
    g = dict(nn={}, plan=[], rounds=0, cost=0.0, cost_expr="", emd=0.0)
    with open(path) as fh:
        for raw in fh:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split(None, 1)
            rest = rest[0] if rest else ""
            if key == "metric":
                metric = rest.strip()
            elif key == "S":
                S.append([float(v) for v in rest.split()])
            elif key == "C":
                C.append([float(v) for v in rest.split()])
            elif key == "nn":
                vals = [int(v) for v in rest.split()]
                g["nn"][vals[0]] = vals[1:]
            elif key == "plan":
                i, j, f = rest.split()
                g["plan"].append((int(i), int(j), float(f)))
            elif key == "rounds":
                g["rounds"] = int(rest)
            elif key == "cost":
                g["cost"] = float(rest)
            elif key == "cost_expr":
                g["cost_expr"] = rest.strip()
            elif key == "emd":
                g["emd"] = float(rest)
            else:
                raise ValueError(f"{path}: unknown record {key}")
    S = np.array(S)
    C = np.array(C)
    return Golden(os.path.basename(path), metric,
                  S[:, :-1].astype(np.float32), S[:, -1].astype(np.float64),
                  C[:, :-1].astype(np.float32), C[:, -1].astype(np.float64), **g)


def all_golden(directory: str) -> list[Golden]:
    return [load(p) for p in sorted(glob.glob(os.path.join(directory, "*.txt")))]
