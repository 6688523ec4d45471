"""FP64 CPU oracle for Priori L+S (arXiv:1411.6206).

Test infrastructure only: imported by tests/, by the smoke check and by the benchmark
CPU-baseline leg. The library never imports it; it shares no code with the CUDA path.
"""
