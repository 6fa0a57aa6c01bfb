"""Reader for the cited fixture files in this folder."""
import os
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_values() -> dict:
    out = {}
    with open(os.path.join(HERE, "paper_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, rest = line.split("=", 1)
            val = rest.split(";", 1)[0].strip()
            try:
                out[key.strip()] = int(val)
            except ValueError:
                try:
                    out[key.strip()] = Fraction(val)
                except ValueError:
                    try:
                        out[key.strip()] = float(val)
                    except ValueError:
                        out[key.strip()] = val
    return out
