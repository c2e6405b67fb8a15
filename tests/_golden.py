"""Reader for the printed values under tests/golden/ (each file cites its source)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def glass_accuracy():
    """{("theta" | "tau_ref", value): {"rays_per_element" | "segments_per_element": x,
    "rms_error": e}} from glass_accuracy.txt."""
    out = {}
    for ln in open(os.path.join(GOLDEN, "glass_accuracy.txt")):
        ln = ln.split("#", 1)[0].split()
        if not ln:
            continue
        key = (ln[0], float(ln[1]))
        out[key] = {ln[i]: float(ln[i + 1]) for i in range(2, len(ln), 2)}
    return out
