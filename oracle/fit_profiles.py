"""Writes the committed Gaussian-mixture profile tables.

Run from the repository root:  python -m oracle.fit_profiles

Part of the FP64 oracle (test infrastructure).  The tables it writes are
inputs shared by the CUDA path and the oracle (both read the same amplitudes
and variances), so parity never depends on fit quality.

Tables (ids as used by the galaxy parameter arrays):
  0  exponential (Sersic n = 1), 6 components;
  1  de Vaucouleurs (n = 4), 10 components;
  2  Sersic grid, nodes n = 0.5 ... 6.0 in steps of 0.25 with K(n) = 8..12
     components (Section 3: the mixture amplitudes and variances vary smoothly
     with n, so a grid of fits is interpolated for intermediate n).

Slots are ordered by decreasing variance.  The Sersic grid is fitted by
continuation from n = 6 downwards, each node starting from the fit at the node
above with its smallest-variance component dropped when K(n) decreases.
Unused slots carry a = 0 and the variance of the same slot at the nearest
higher node, so that interpolating a linearly and log v linearly in n is
continuous across nodes.
"""

import json
import os
import sys

import numpy as np

from .sersic import fit_error, fit_mog, sersic_k

K_MAX = 12
OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "workloads", "mog_profiles.json")


def sersic_components(n):
    """Number of active mixture components at a Sersic grid node."""
    if n <= 1.0:
        return 8
    if n <= 2.0:
        return 9
    if n <= 3.0:
        return 10
    if n <= 4.5:
        return 11
    return 12


def _pad(a, v, fill_v):
    ap = np.zeros(K_MAX)
    vp = np.array(fill_v, dtype=np.float64).copy()
    ap[:len(a)] = a
    vp[:len(v)] = v
    return ap, vp


def fixed_table(tid, name, n, k):
    a, v = fit_mog(n, k)
    l2, half = fit_error(n, a, v)
    ap, vp = _pad(a, v, np.full(K_MAX, v[-1]))
    return dict(id=tid, name=name, nodes=[n], k=[k], amp=ap.tolist(), var=vp.tolist(),
                fit=dict(k_n=sersic_k(n), rel_l2=[l2], light_within_re=[half]))


def sersic_table(tid=2):
    nodes = np.round(np.arange(0.5, 6.0 + 1e-9, 0.25), 2)
    fits = {}
    init = None
    for n in nodes[::-1]:
        k = sersic_components(n)
        if init is not None and len(init[0]) > k:
            init = (init[0][:k], init[1][:k])
        a, v = fit_mog(float(n), k, init=init)
        fits[n] = (a, v)
        init = (a, v)
        print(f"  n={n:4.2f} K={k:2d} rel_l2={fit_error(n, a, v)[0]:.3e}", file=sys.stderr)
    amp, var, ks, l2s, halves = [], [], [], [], []
    fill = None
    for n in nodes[::-1]:
        a, v = fits[n]
        if fill is None:
            fill = np.full(K_MAX, v[-1])
        ap, vp = _pad(a, v, fill)
        fill = vp
        amp.append(ap)
        var.append(vp)
        ks.append(len(a))
        l2, half = fit_error(n, a, v)
        l2s.append(l2)
        halves.append(half)
    rev = slice(None, None, -1)
    return dict(id=tid, name="sersic", nodes=nodes.tolist(), k=ks[rev],
                amp=np.array(amp[rev]).ravel().tolist(), var=np.array(var[rev]).ravel().tolist(),
                fit=dict(k_n=[sersic_k(n) for n in nodes], rel_l2=l2s[rev], light_within_re=halves[rev]))


def main(out=OUT):
    tables = [fixed_table(0, "exp", 1.0, 6), fixed_table(1, "dev", 4.0, 10), sersic_table(2)]
    doc = dict(
        description="Gaussian-mixture approximations of unit-flux Sersic profiles in r_e units: "
                    "sum_i amp_i N(0, var_i I), sum amp = 1; slots ordered by decreasing var; "
                    "amp/var are row-major [node][12].",
        method="weighted least squares over 1e-4 < r <= 8 r_e, weight 2 pi r dr; written by oracle/fit_profiles.py",
        k_max=K_MAX, tables=tables)
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    print(f"wrote {out}", file=sys.stderr)


if __name__ == "__main__":
    main()
