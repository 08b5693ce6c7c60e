// Instantiation of the hot-path kernels for chains of length 1.
#include "mpg_kernels_impl.cuh"

template struct mpg::KLaunch<1>;
