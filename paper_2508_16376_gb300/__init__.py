"""GB300-native cycle-based RTL stuck-at fault simulation (the hot path of RIROS,
arXiv 2508.16376): good-machine trace, sparse-diff faulty machines, output compare and
fault dropping, all in hand-written sm_103a CUDA kernels behind the C-ABI library
`librtlfs` (include/rtlfs.h). `rtlfs` is the thin ctypes binding; `synth` builds seeded
synthetic workloads. Submodules are imported lazily so that loading `synth` never loads
the CUDA library."""
