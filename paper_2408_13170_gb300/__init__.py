"""GB300-native evaluation of the semi-coherent search statistic Upsilon_N
(Bandopadhyay & Moore, arXiv:2408.13170).

``scstat`` binds the CUDA library's C ABI (include/scstat.h); ``synth``
draws seeded synthetic inputs shaped like the paper's mock LISA streams.
"""
