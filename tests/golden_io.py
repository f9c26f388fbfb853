"""Readers of the fixtures under tests/golden/ (values printed in the paper)."""
import math
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def cnot_unitary() -> np.ndarray:
    """The Ralph CNOT unitary printed in Sec. 3.3 (Figure ralph_cnot_unitary)."""
    rows = []
    for line in open(os.path.join(GOLD, "cnot_unitary.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([complex(eval(e.strip(), {"sqrt": math.sqrt, "j": 1j})) for e in line.split("|")])
    return np.array(rows)
