"""Independent FP64 CPU oracle of the wave-tank step -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It shares no code with the CUDA library under
``paper_2206_07732_gb300/``; the two meet only through the seeded inputs of
``paper_2206_07732_gb300.synth``.
"""
