"""Record an observed agreement beside the bound a test asserts.

Each call prints one line ``OBSERVED <name> <value> <bound>`` (shown with
pytest -s) and, when the environment variable MT_OBSERVE names a file,
appends the same as a JSON line there.  The bounds of the GPU parity tests
are stated multiples of the values observed on GB300; this keeps the
observed values visible on every run.
"""
import json
import os


def observe(name: str, value: float, bound: float) -> None:
    print("OBSERVED %s %.3e %.3e" % (name, float(value), float(bound)))
    path = os.environ.get("MT_OBSERVE")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"name": name, "value": float(value), "bound": float(bound)}) + "\n")
