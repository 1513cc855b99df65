"""GB300-native short-range tree / FMM gravity after GADGET-4 (Springel et al. 2021).

The compute path is the sm_103a CUDA library ``libg4.so`` behind the C ABI in
``include/g4.h``; ``paper_2010_03567_gb300.g4`` is its thin Python binding (argument
marshalling only) and ``synth`` holds the seeded synthetic particle sets.
"""
