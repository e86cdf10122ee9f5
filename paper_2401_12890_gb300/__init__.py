"""GB300-native LADMM for spatial-spectral partial-volume compartment mapping.

The solver is a C-ABI CUDA library (include/ssm.h, sources in csrc/) for sm_103a;
`paper_2401_12890_gb300.ssm` is its thin ctypes binding and `synth` builds seeded
synthetic inputs shaped like the paper's experiments.
"""
