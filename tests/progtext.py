"""Text form of postfix programs for tests: "x0 c1 * sin" -> uint8 tokens."""
import numpy as np

OPS = {"+": 0, "-": 1, "*": 2, "/": 3, "sin": 4, "cos": 5, "exp": 6, "log": 7, "sqrt": 8, "sq": 9,
       "inv": 10, "tan": 11, "asin": 12, "acos": 13, "atan": 14, "tanh": 15}
NAMES = {v: k for k, v in OPS.items()}


def parse(text: str) -> np.ndarray:
    out = []
    for w in text.split():
        if w in OPS:
            out.append(OPS[w])
        elif w[0] == "x":
            out.append(16 + int(w[1:]))
        elif w[0] == "c":
            out.append(32 + int(w[1:]))
        else:
            raise ValueError(w)
    return np.array(out, np.uint8)


def show(tokens) -> str:
    out = []
    for t in tokens:
        t = int(t)
        if t in NAMES:
            out.append(NAMES[t])
        elif 16 <= t < 32:
            out.append(f"x{t - 16}")
        elif 32 <= t < 48:
            out.append(f"c{t - 32}")
        else:
            out.append(f"?{t}")
    return " ".join(out)


def pack(programs, Lmax=None):
    """List of token arrays -> ([P, Lmax] uint8, lengths int32)."""
    Lmax = Lmax or max(len(p) for p in programs)
    arr = np.zeros((len(programs), Lmax), np.uint8)
    lens = np.zeros(len(programs), np.int32)
    for i, p in enumerate(programs):
        arr[i, : len(p)] = p
        lens[i] = len(p)
    return arr, lens


def load_hand_cases(path):
    import math  # noqa: F401  (used by eval of the expected column)
    cases = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        prog, consts, xs, expect = [s.strip() for s in line.split("|")]
        c = [float(v) for v in consts.split()] if consts else []
        x = [float(v) for v in xs.split()]
        cases.append((prog, c, x, eval(expect, {"math": math})))
    return cases
