"""ASH parallel spatial hashing on GB300 (sm_103a).

The hash map lives behind the C ABI in include/ash.h (libash.so, built from
csrc/); `paper_2110_00511_gb300.ash` is the thin ctypes binding with the same
names.  `workloads` holds the seeded synthetic input generators.
"""
__all__ = ["ash", "workloads"]
