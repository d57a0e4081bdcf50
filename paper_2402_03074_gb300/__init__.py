"""GB300-native HWENO-U hot path (arXiv 2402.03074): CUDA kernels for sm_103a behind a C ABI."""
