"""Write the oracle's FCF pole/weight tables (Algorithm 2) to oracle/tables/.

ORACLE -- test infrastructure only.  Calls nothing but ``oracle``.

    python -m oracle.make_tables            # the default set
    python -m oracle.make_tables 16 24      # one (K, R1) pair
"""

from __future__ import annotations

import os
import sys
import time

from . import fcf, tables

# (K, R1) pairs used by the tests, the smoke check and the benchmark workloads.
DEFAULT_SET = [(8, 8), (12, 14), (16, 10), (16, 24), (32, 68), (64, 162)]


def write(K, R1):
    t0 = time.time()
    sigma, beta, info = fcf.faber_cf(R1, K)
    path = tables.table_path(K, R1)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write(tables.format_table(K, R1, sigma, beta, info))
    print("wrote %s (L=%d, %.1fs)" % (path, info["L"], time.time() - t0), flush=True)


def main(argv):
    if len(argv) == 2:
        pairs = [(int(argv[0]), float(argv[1]))]
    else:
        pairs = DEFAULT_SET
    for K, R1 in pairs:
        write(K, R1)


if __name__ == "__main__":
    main(sys.argv[1:])
