"""GB300 (sm_103a) implementation of the FFT-accelerated shifted-Green-function Nystrom operator of
Bruno & Maas (arXiv:1707.04950). The compute path lives in the CUDA library built from csrc/ and is
reached through the C ABI of include/sgf.h; `sgf` is its ctypes binding, `inputs` the seeded
synthetic workloads."""
