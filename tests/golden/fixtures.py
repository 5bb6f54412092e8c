"""Readers for the hand-worked fixtures (hand_worked.txt, setcover_hand.txt)."""
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


def load_setcover(path=os.path.join(HERE, "setcover_hand.txt")):
    """Blocks of setcover_hand.txt: n, eps_ppm, priorities, edges (u, v), expected step
    of each set, expected number of steps."""
    out, cur = [], None
    for raw in open(path):
        line = raw.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0] == "graph":
            kv = dict(t.split("=") for t in tok[2:])
            cur = dict(name=tok[1], n=int(kv["n"]), eps_ppm=int(kv["eps_ppm"]), edges=[])
        elif tok[0] == "pri":
            cur["pri"] = [int(x) for x in tok[1:]]
        elif tok[0] == "edge":
            cur["edges"].append((int(tok[1]), int(tok[2])))
        elif tok[0] == "expect":
            cur["expect"] = [int(x) for x in tok[1:]]
        elif tok[0] == "steps":
            cur["steps"] = int(tok[1])
        elif tok[0] == "end":
            out.append(cur)
            cur = None
    return out
