"""FCF pole/weight tables of the oracle.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

``poles(K, R1)`` returns (sigma, beta, meta) for exp on i[-R1, R1]
(Algorithm 2).  The values come from ``oracle.fcf`` at 60 significant digits;
because mpmath is not installed on every host, each table is computed once by
``oracle/make_tables.py`` and stored as text in ``oracle/tables/`` (30
significant digits per entry).  When a table is missing and mpmath is present
it is computed on the fly.
"""

from __future__ import annotations

import os

import numpy as np

_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tables")


def table_path(K, R1):
    return os.path.join(_DIR, "fcf_K%d_R%s.txt" % (int(K), ("%g" % float(R1)).replace(".", "p")))


def format_table(K, R1, sigma, beta, info):
    import mpmath as mp
    lines = [
        "# FCF poles/weights of exp on i[-R1,R1] (Algorithm 2), written by oracle/make_tables.py",
        "K %d" % K,
        "R1 %s" % mp.nstr(mp.mpf(R1), 20),
        "L %d" % info["L"],
        "sigma_K+1 %s" % mp.nstr(info["sigma"], 25),
        "# re(sigma_j) im(sigma_j) re(beta_j) im(beta_j) re(z_j) im(z_j)",
    ]
    for s, b, zz in zip(sigma, beta, info["z"]):
        lines.append(" ".join(mp.nstr(x, 30, min_fixed=1, max_fixed=0)
                              for x in (mp.re(s), mp.im(s), mp.re(b), mp.im(b), mp.re(zz), mp.im(zz))))
    return "\n".join(lines) + "\n"


def parse_table(text):
    meta = {}
    rows = []
    for line in text.splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] in ("K", "L"):
            meta[parts[0]] = int(parts[1])
        elif parts[0] in ("R1", "sigma_K+1"):
            meta[parts[0]] = float(parts[1])
        else:
            rows.append([float(p) for p in parts])
    rows = np.array(rows)
    sigma = rows[:, 0] + 1j * rows[:, 1]
    beta = rows[:, 2] + 1j * rows[:, 3]
    meta["z"] = rows[:, 4] + 1j * rows[:, 5]
    return sigma, beta, meta


def poles(K, R1):
    """(sigma, beta, meta) as complex128 numpy arrays."""
    p = table_path(K, R1)
    if os.path.exists(p):
        with open(p) as f:
            return parse_table(f.read())
    from . import fcf  # needs mpmath
    sigma, beta, info = fcf.faber_cf(R1, K)
    return parse_table(format_table(K, R1, sigma, beta, info))
