"""GB300-native batched pair-interaction engine after the G-Charm runtime
strategies (Rengasamy & Vadhiyar, arXiv 2008.05712): kernel combining,
chare-table data reuse, sorted coalescing pack, Barnes-Hut gravity and
cell-pair Lennard-Jones tasks.  The compute path is libgcharm.so (CUDA,
sm_103a, C ABI in include/gcharm.h); ``gcharm`` is its Python binding.
"""
