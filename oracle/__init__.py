"""Plain FP64 CPU oracle of YAND-MVSK.  Test infrastructure only: imported by
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs."""
