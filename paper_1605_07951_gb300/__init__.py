"""GB300 resolvent sampling (RSRR hot path) behind the C ABI of include/rsrr.h.

`from paper_1605_07951_gb300 import rsrr` loads librsrr.so (built in tree by
__graft_entry__.build()); there is no CPU fallback.
"""
