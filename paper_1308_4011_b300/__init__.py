"""B300-native Move Method metric engine (LCOM, CBO, fan-in/out and
incremental move evaluation), after Napoli, Pappalardo and Tramontana,
"Using Modularity Metrics to assist Move Method Refactoring of Large Systems"
(CISIS 2013).

Submodules are imported lazily: ``synth`` (seeded input generator) needs only
gcc, ``mmref`` (the CUDA library binding) needs the built ``libmmref.so``.
"""
__all__ = ["synth", "mmref"]
