"""Reader of the printed-value fixtures under tests/golden/ (whitespace-separated rows;
lines starting with '#' hold the citation and column meanings)."""
from pathlib import Path

GOLDEN = Path(__file__).resolve().parent / "golden"


def rows(name):
    """The fixture's data rows as lists of strings (numbers stay strings so that a test
    can read how many digits were printed)."""
    out = []
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out
