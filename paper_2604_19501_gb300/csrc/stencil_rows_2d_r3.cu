// Assembled-stencil row kernels for 2D, radius 3.
#include "stencil_rows.cuh"

namespace helm {
template int stencil_rows<2, 3>(Prec, const GridDims&, const void*, const void*, int, Prec, const void*,
                                 const void*, void*, int, double, int, cudaStream_t);
}  // namespace helm
