"""Reader of the hand-worked fixtures in tests/golden/*.txt."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    rec = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(":")
            rec[key.strip()] = val.strip()
    out = {"input": rec["input_ascii"].encode("ascii")}
    for key in ("counts", "lengths"):
        out[key] = {int(k): int(v) for k, v in (t.split("=") for t in rec[key].split())}
    out["codes"] = {int(k): v for k, v in (t.split("=") for t in rec["codes"].split())}
    out["total_bits"] = int(rec["total_bits"])
    out["words"] = [int(w, 16) for w in rec["payload_words_hex"].split()]
    out["chunk_symbols"] = int(rec["chunk_symbols"])
    out["offsets"] = [int(v) for v in rec["offsets"].split()]
    return out


def all_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
