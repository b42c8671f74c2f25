// Element kernels instantiated for k = 3 (q = 4 and 5).
#include "k_element.cuh"
HD_DEFINE_K(3)
