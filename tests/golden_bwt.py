"""Reader of the block-sorting fixtures in tests/golden/bwt/*.txt."""
import os

GOLDEN_BWT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bwt")


def load(name):
    rec = {}
    with open(os.path.join(GOLDEN_BWT, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(":")
            rec[key.strip()] = val.strip()
    return {
        "input": rec["input_ascii"].encode("ascii"),
        "block": int(rec["block"]),
        "last": rec["last_ascii"].encode("ascii"),
        "primary": [int(v) for v in rec["primary"].split()],
    }


def all_names():
    return sorted(f for f in os.listdir(GOLDEN_BWT) if f.endswith(".txt"))
