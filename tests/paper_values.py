"""Reader of the paper's printed values stored under tests/golden/.

Each fixture is a text file: '#' lines carry the citation and the meaning of each
key; every other line is a key followed by one or more numbers.
"""
from pathlib import Path

GOLDEN = Path(__file__).resolve().parent / "golden"


def load(name: str) -> dict:
    """{key: float} for one-number keys, {key: [floats]} for the others."""
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        nums = [float(v) for v in vals]
        out[key] = nums[0] if len(nums) == 1 else nums
    return out
