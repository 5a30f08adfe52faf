"""Loader for the committed Gaussian-mixture profile tables.

Each table approximates a unit-flux radial profile (in units of the effective
radius) by sum_i a_i N(0, v_i I) with sum_i a_i = 1 (Section 1, footnote on
mixtures).  A table has one or more nodes in Sersic index n; each node stores
``K_MAX`` slots of (a_i, v_i), unused slots having a_i = 0.  Fixed profiles
(exponential, de Vaucouleurs) have a single node; the Sersic table has a grid
of nodes between which a_i and log v_i are interpolated linearly in n
(Section 3, Sersic interpolation).

The values are written by the oracle's least-squares fitter and committed as
``mog_profiles.json`` beside this file; this module only reads them.
"""

import json
import os
from dataclasses import dataclass

import numpy as np

K_MAX = 12
TABLE_PATH = os.path.join(os.path.dirname(__file__), "mog_profiles.json")


@dataclass
class ProfileTable:
    name: str
    nodes: np.ndarray   # (n_nodes,) float64 Sersic index of each node
    amp: np.ndarray     # (n_nodes, K_MAX) float64
    var: np.ndarray     # (n_nodes, K_MAX) float64, variance in r_e^2 units
    k: np.ndarray       # (n_nodes,) active components per node


def load_profile_tables(path=TABLE_PATH):
    """Returns {profile_id: ProfileTable}."""
    with open(path) as f:
        doc = json.load(f)
    out = {}
    for t in doc["tables"]:
        out[int(t["id"])] = ProfileTable(
            name=t["name"],
            nodes=np.array(t["nodes"], dtype=np.float64),
            amp=np.array(t["amp"], dtype=np.float64).reshape(-1, K_MAX),
            var=np.array(t["var"], dtype=np.float64).reshape(-1, K_MAX),
            k=np.array(t["k"], dtype=np.int64),
        )
    return out
