"""The autotuner's chosen launch configuration per workload (tuned.json beside this file,
written by `python -m paper_2302_08252_gb300.autotune --write-tuned` on a GB300).  The
bench and the serving loop take their defaults from it, so that what they time is what
the autotuner picked."""
from __future__ import annotations

import json
import os

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
KEYS = ("form", "layout", "block_size", "driver")


def load(path: str = PATH) -> dict:
    with open(path) as f:
        return json.load(f)


def config(workload: str, path: str = PATH) -> dict | None:
    """{"form", "layout", "block_size", "driver"} for the workload, or None if not tuned."""
    entry = load(path).get(workload)
    return None if entry is None else {k: entry[k] for k in KEYS}


def write(workload: str, best: dict, tuned_on: str, command: str, path: str = PATH) -> None:
    data = load(path) if os.path.exists(path) else {}
    data[workload] = {**{k: best[k] for k in KEYS}, "tuned_on": tuned_on, "command": command}
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
        f.write("\n")
