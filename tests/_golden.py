"""Parser for the hand-derived task-graph fixture in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_MODES = {"R": 0, "W": 1, "C": 2, "A": 3, "M": 4}


def load_dag_fixture(name="dag_modes_small.txt"):
    tasks, keys, modes = [], [], []
    edges, indeg = [], None
    keymap = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("task"):
                head, body = line.split(":", 1)
                t = int(head.split()[1])
                for acc in body.split(","):
                    m, k = acc.split()
                    keymap.setdefault(k, len(keymap))
                    tasks.append(t)
                    keys.append(keymap[k])
                    modes.append(_MODES[m])
            elif line.startswith("edges:"):
                for e in line.split(":", 1)[1].split():
                    u, v = e.split("-")
                    edges.append((int(u), int(v)))
            elif line.startswith("indeg:"):
                indeg = [int(x) for x in line.split(":", 1)[1].split()]
    ntasks = max(tasks) + 1
    return (ntasks, np.asarray(tasks, np.uint32), np.asarray(keys, np.uint64),
            np.asarray(modes, np.int32), edges, indeg)
