"""Readers for the text fixtures under tests/golden (values printed in the paper)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].strip()
            if ln:
                yield ln.split()


def worked_examples():
    out = []
    for tok in _lines("worked_examples.txt"):
        name, n, t, ctrl, what, vals = tok
        out.append(dict(name=name, n=int(n), target=int(t),
                        controls=[int(c) for c in ctrl.split(",")],
                        what=what, vals=[int(v) for v in vals.split(",")]))
    return out


def parse_swaps(spec_tokens):
    """'0:2' -> one step with one pair; '0:2,1:3' -> one step with two pairs."""
    steps = []
    for tok in spec_tokens:
        if tok == "-":
            continue
        steps.append([tuple(int(x) for x in p.split(":")) for p in tok.split(",")])
    return steps


def layout_table_steps(name):
    steps, body = {}, {}
    for tok in _lines(name):
        if not (len(tok) == 6 and all(c in "01" for c in tok[1])):
            steps[tok[0]] = parse_swaps(tok[1:])
        else:
            sig, addr = tok[0], int(tok[1], 2)
            for R, logical in enumerate(tok[2:]):
                body.setdefault(sig, {})[R * 4 + addr] = int(logical, 2)
    return steps, body


def shor_table(name="shortab_L24.txt"):
    d = {}
    for tok in _lines(name):
        if tok[0] == "Q":
            d["Q"] = [float(v) for v in tok[1:]]
        else:
            d[tok[0]] = int(tok[1])
    return d


def adders():
    out = []
    for tok in _lines("adders.txt"):
        name, m, vals, no = tok
        out.append(dict(name=name, m=int(m), values=[int(v) for v in vals.split(",")],
                        n_ops=None if no == "-" else int(no)))
    return out
