"""Reader for paper_tables.txt (values printed in the paper's Section 3 tables)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    rows = {}
    with open(os.path.join(HERE, "paper_tables.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = [float(v) for v in vals]
    return rows
