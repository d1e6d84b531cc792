// Assembled-stencil row kernels for 3D, radius 1.
#include "stencil_rows.cuh"

namespace helm {
template int stencil_rows<3, 1>(Prec, const GridDims&, const void*, const void*, int, Prec, const void*,
                                 const void*, void*, int, double, int, cudaStream_t);
}  // namespace helm
