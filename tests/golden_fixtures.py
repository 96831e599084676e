"""Reader of the small text fixtures under tests/golden/: one ``key = value``
per line, ``#`` starts a comment.  Each fixture holds values printed in the
paper for one of its worked examples, with the passage cited in its header."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, value = (x.strip() for x in line.split("=", 1))
            out[key] = int(value) if value.lstrip("-").isdigit() else float(value)
    return out
