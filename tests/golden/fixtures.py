"""Reader for the hand-worked fixtures in hand_worked.txt."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
INF = 0xFFFFFFFF


def load(path=os.path.join(HERE, "hand_worked.txt")):
    out, cur = [], None
    for raw in open(path):
        line = raw.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "graph":
            kv = dict(t.split("=") for t in tok[2:])
            cur = dict(name=tok[1], n=int(kv["n"]), src=int(kv["src"]),
                       target=int(kv["target"]) if "target" in kv else None, edges=[])
        elif tok[0] == "edge":
            cur["edges"].append(tuple(int(x) for x in tok[1:4]))
        elif tok[0] == "expect":
            cur["expect"] = [INF if x == "inf" else int(x) for x in tok[1:]]
        elif tok[0] == "end":
            out.append(cur)
            cur = None
    return out
