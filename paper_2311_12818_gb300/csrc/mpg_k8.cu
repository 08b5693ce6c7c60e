// Instantiation of the hot-path kernels for chains of length 8.
#include "mpg_kernels_impl.cuh"

template struct mpg::KLaunch<8>;
