"""GB300-native PCF Learned Sort.

The sort runs in hand-written CUDA kernels behind the C ABI declared in
include/pcfsort.h; `paper_2405_07122_gb300.pcfsort` is the thin Python
binding (argument marshalling only).  `workloads` draws the seeded
synthetic inputs.  Submodules are imported explicitly so that importing
the input generators does not load the CUDA library.
"""
