// Element kernels instantiated for k = 5 (q = 6 and 7).
#include "k_element.cuh"
HD_DEFINE_K(5)
