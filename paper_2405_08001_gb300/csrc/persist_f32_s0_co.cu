// The FP32 form's corotated densities (FCR, ARAP): the persistent time step in the default block shape, in a
// translation unit of its own (persist_shapes.cuh).
#include "persist_shapes.cuh"

namespace pncg {
cudaError_t persist_launch_corot(const Dev<float> &D, const BPDev &B, const PersistArgs &A, int grid, cudaStream_t s)
{
    Dev<float> d = D;
    BPDev b = B;
    PersistArgs a = A;
    void *args[] = {(void *)&d, (void *)&b, (void *)&a};
    return cudaLaunchCooperativeKernel((const void *)k_persistent<float, PSHAPE_PB[0], PSHAPE_MINB[0], true>, dim3(grid),
                                       dim3(PSHAPE_PB[0]), args, 0, s);
}
cudaError_t persist_occupancy_corot(int *per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_persistent<float, PSHAPE_PB[0], PSHAPE_MINB[0], true>,
                                                         PSHAPE_PB[0], 0);
}
}
