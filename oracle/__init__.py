"""CPU oracle for Rejection-Free Partial Neighbor Search (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this package.  The product (paper_2210_10513_gb300) never does.
"""
