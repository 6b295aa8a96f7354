"""FP64 CPU oracle of SegSALSA-STR. Test infrastructure only: imported by tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline legs, never by the product path."""
