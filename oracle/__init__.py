"""FP64 CPU oracle for MC-moments micro-macro Parareal (arXiv 2310.11365).

Test infrastructure only: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may use it; the product path never does.
"""
from .oracle import *  # noqa: F401,F403
