"""Reader for the small text fixtures in this folder (values printed in the
paper, each file citing the table it comes from)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def read_table(name):
    """Return {row_name: [value, value]} from a two-column fixture file."""
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            out[parts[0]] = [float(v) for v in parts[1:]]
    return out
