"""FP64 CPU oracle for Priori L+S (arXiv:1411.6206).

Test infrastructure only: imported by tests/, by __graft_entry__.smoke() and by bench.py's
CPU-baseline leg. The library never imports it; it shares no code with the CUDA path.
"""
