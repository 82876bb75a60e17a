"""Shared helpers for the tests (no decomposition arithmetic here)."""

import os
import re
import threading

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_lock = threading.Lock()


def ensure_built():
    """Build the CUDA library once per session if it is missing."""
    from paper_1806_07985_gb300 import build, nncp
    with _lock:
        if not os.path.exists(nncp.LIB_PATH):
            build.build()
    return nncp.load()


def header_functions():
    """Names of every function declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(nncp_\w+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
