"""Published reference values for the oracle's pins, read from
tests/golden/published_constants.txt (each line carries its source)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "published_constants.txt")


def _load():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


VALUES = _load()


def published(name: str) -> float:
    return VALUES[name]
