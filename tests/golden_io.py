"""Readers of the text fixtures under tests/golden/ (no codec arithmetic)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_tables():
    """{'time': [(table, image, w, h, cpu_ms, gpu_ms)], 'psnr': [(table, image, w, h, dct_db, cordic_db)]}"""
    out = {"time": [], "psnr": []}
    for line in open(os.path.join(GOLDEN, "paper_tables.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        kind, table, image, w, h, a, b = line.split()
        out[kind].append((int(table), image, int(w), int(h), float(a), float(b)))
    return out


def worked_blocks():
    """[{'name', 'quality', 'chroma', 'sample', 'Q', 'Y', 'q', 'recon' (8x8 int64), 'sse'}]"""
    blocks, cur = [], None
    for line in open(os.path.join(GOLDEN, "worked_blocks.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "block":
            cur = {"name": f[1], "quality": int(f[3]), "chroma": f[4] == "chroma"}
            blocks.append(cur)
        elif f[0] == "sse":
            cur["sse"] = int(f[1])
        else:
            cur.setdefault(f[0], []).append([int(v) for v in f[1:]])
    for b in blocks:
        for k in ("sample", "Q", "Y", "q", "recon"):
            b[k] = np.array(b[k], dtype=np.int64)
    return blocks
