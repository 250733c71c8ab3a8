"""Readers for the fixtures under tests/golden (values typed from the paper)."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_matrix(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def load_symbolic(name, **values):
    """Evaluate the named printed vector of symbolic_vectors.txt at the given values."""
    with open(os.path.join(GOLDEN, "symbolic_vectors.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, _cite, body = [s.strip() for s in line.split("|")]
            if key == name:
                env = {"__builtins__": {}}
                env.update(values)
                return np.array([float(eval(e, env)) for e in body.split(",")])
    raise KeyError(name)


def paper_numbers():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as fh:
        return json.load(fh)
