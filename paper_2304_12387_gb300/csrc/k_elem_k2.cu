// Element kernels instantiated for k = 2 (q = 3 and 4).
#include "k_element.cuh"
HD_DEFINE_K(2)
