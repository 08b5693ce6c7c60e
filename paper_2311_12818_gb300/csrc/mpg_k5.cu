// Instantiation of the hot-path kernels for chains of length 5.
#include "mpg_kernels_impl.cuh"

template struct mpg::KLaunch<5>;
