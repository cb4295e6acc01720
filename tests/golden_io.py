"""Parser for the worked-example fixtures under tests/golden/."""
from __future__ import annotations

import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    d = {"reads": [], "nodes": [], "edges": [], "unitigs": [], "paper": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, *rest = line.split()
            if tag == "k":
                d["k"] = int(rest[0])
            elif tag == "read":
                d["reads"].extend(rest)
            elif tag == "node":
                d["nodes"].append(rest[0])
            elif tag == "edge":
                s, t, o1, o2, m = rest
                d["edges"].append((s, t, int(o1), int(o2), int(m)))
            elif tag == "unitig":
                d["unitigs"].append(rest[0])
            elif tag.startswith("paper_"):
                d["paper"].append((tag[len("paper_"):], rest))
            else:
                raise ValueError(f"{name}: unknown tag {tag}")
    return d


def all_fixtures() -> list[str]:
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
