"""CPU oracle of the SpeedyGS decode path -- TEST INFRASTRUCTURE ONLY.

Used by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``, and
by nothing else.  It shares no code with the CUDA library and imports nothing from it.
Every function is pinned by tests against what the paper and mathematics fix (round trips,
closed forms, brute force, brute-force enumeration); see the test files.
"""
