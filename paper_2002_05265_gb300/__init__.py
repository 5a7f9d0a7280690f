"""GB300-native D2Q9 stream-and-collide lattice Boltzmann kernels for every collision model
compared by Coreixas, Wissocq, Chopard & Latt (arXiv:2002.05265).

The compute path is the CUDA shared library `liblbm.so` (C ABI declared in include/lbm.h);
`paper_2002_05265_gb300.lbm` is its thin ctypes binding.  Importing this package does not
load the library; the binding loads it on first use and raises if it is missing.
"""
