"""FP64 CPU oracle of the specular ray-tracing path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
legs may import this package. It shares no code with the CUDA library.
"""
