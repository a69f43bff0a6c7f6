// Block shapes of the persistent time step.  Each shape (threads per block, blocks per SM) is an instantiation of
// k_persistent compiled in a translation unit of its own (persist_<precision>_s<n>.cu, built in parallel); the
// host picks one per handle, fixed (sim_options.block_shape >= 0) or by timing one time step in each
// (block_shape = -1, the block-shape autotuner).
#pragma once

#include "persistent.cuh"

namespace pncg {

constexpr int N_PSHAPES = 5;
// shape s: PSHAPE_PB[s] threads per block, at most PSHAPE_MINB[s] blocks per SM (the launch bound the compiler
// fits the registers to: 128 per thread at 2 x 256, 85 at 3 x 256, 255 at 1 x 256; 128 at 1 x 512, 168 at 1 x 384)
constexpr int PSHAPE_PB[N_PSHAPES] = {256, 512, 256, 256, 384};
constexpr int PSHAPE_MINB[N_PSHAPES] = {2, 1, 3, 1, 1};

// launch of shape S (cooperative, grid blocks, PSHAPE_PB[S] threads) and its occupancy (blocks per SM)
template <typename R, int S> cudaError_t persist_launch(const Dev<R> &D, const BPDev &B, const PersistArgs &A, int grid,
                                                        cudaStream_t s);
template <typename R, int S> cudaError_t persist_occupancy(int *per_sm);

#define PNCG_PERSIST_DECL(R, S)                                                                                 \
    template <> cudaError_t persist_launch<R, S>(const Dev<R> &, const BPDev &, const PersistArgs &, int,       \
                                                 cudaStream_t);                                                \
    template <> cudaError_t persist_occupancy<R, S>(int *);
PNCG_PERSIST_DECL(float, 0) PNCG_PERSIST_DECL(float, 1) PNCG_PERSIST_DECL(float, 2) PNCG_PERSIST_DECL(float, 3)
PNCG_PERSIST_DECL(float, 4)
PNCG_PERSIST_DECL(double, 0) PNCG_PERSIST_DECL(double, 1) PNCG_PERSIST_DECL(double, 2) PNCG_PERSIST_DECL(double, 3)
PNCG_PERSIST_DECL(double, 4)
#undef PNCG_PERSIST_DECL

// the definitions, one shape per translation unit
#define PNCG_PERSIST_DEF(R, S)                                                                                  \
    template <> cudaError_t persist_launch<R, S>(const Dev<R> &D, const BPDev &B, const PersistArgs &A, int grid, \
                                                 cudaStream_t s)                                               \
    {                                                                                                          \
        Dev<R> d = D;                                                                                          \
        BPDev b = B;                                                                                           \
        PersistArgs a = A;                                                                                     \
        void *args[] = {(void *)&d, (void *)&b, (void *)&a};                                                   \
        return cudaLaunchCooperativeKernel((const void *)k_persistent<R, PSHAPE_PB[S], PSHAPE_MINB[S]>,         \
                                           dim3(grid), dim3(PSHAPE_PB[S]), args, 0, s);                        \
    }                                                                                                          \
    template <> cudaError_t persist_occupancy<R, S>(int *per_sm)                                               \
    {                                                                                                          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_persistent<R, PSHAPE_PB[S], PSHAPE_MINB[S]>, \
                                                             PSHAPE_PB[S], 0);                                 \
    }

// The FP32 form's corotated densities (FCR, ARAP) run their own instantiation (the Neo-Hookean kernels carry none
// of their code and registers), in the default shape only.
cudaError_t persist_launch_corot(const Dev<float> &D, const BPDev &B, const PersistArgs &A, int grid, cudaStream_t s);
cudaError_t persist_occupancy_corot(int *per_sm);

// run-time dispatch over the shapes
template <typename R>
inline cudaError_t persist_launch_shape(int shape, const Dev<R> &D, const BPDev &B, const PersistArgs &A, int grid,
                                        cudaStream_t s)
{
    switch (shape) {
    case 1: return persist_launch<R, 1>(D, B, A, grid, s);
    case 2: return persist_launch<R, 2>(D, B, A, grid, s);
    case 3: return persist_launch<R, 3>(D, B, A, grid, s);
    case 4: return persist_launch<R, 4>(D, B, A, grid, s);
    default: return persist_launch<R, 0>(D, B, A, grid, s);
    }
}
template <typename R> inline cudaError_t persist_occupancy_shape(int shape, int *per_sm)
{
    switch (shape) {
    case 1: return persist_occupancy<R, 1>(per_sm);
    case 2: return persist_occupancy<R, 2>(per_sm);
    case 3: return persist_occupancy<R, 3>(per_sm);
    case 4: return persist_occupancy<R, 4>(per_sm);
    default: return persist_occupancy<R, 0>(per_sm);
    }
}

} // namespace pncg
