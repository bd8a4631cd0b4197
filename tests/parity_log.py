"""Achieved errors of the parity tests against the FP64 oracle, one record per comparison.

The records are printed as a table at the end of the pytest run (tests/conftest.py) and, when
IRLS_PARITY_JSON names a file, appended to it as JSON lines, so that every bar and every
allowance a test used can be audited next to the error it measured."""
from __future__ import annotations

import json
import os

RECORDS: list[dict] = []


def record(**kw) -> dict:
    RECORDS.append(kw)
    path = os.environ.get("IRLS_PARITY_JSON")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(kw, default=float) + "\n")
    return kw


def table() -> list[str]:
    if not RECORDS:
        return []
    lines = [f"{'case':<58} {'max|dU|':>9} {'U bar':>8} {'dL1/L1':>9} {'L1 bar/L1':>9} "
             f"{'K agree':>8}  bars"]
    for r in RECORDS:
        lines.append(f"{r['case'][:58]:<58} {r['err_u']:9.2e} {r['atol']:8.1e} "
                     f"{r['dl1_rel']:9.2e} {r['l1_bar_rel']:9.2e} {r['k_agree']:8.5f}  "
                     f"{r['bars']}")
    return lines
