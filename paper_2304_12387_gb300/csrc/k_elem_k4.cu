// Element kernels instantiated for k = 4 (q = 5 and 6).
#include "k_element.cuh"
HD_DEFINE_K(4)
