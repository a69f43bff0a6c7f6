// sim_pHp_noalloc: an allocation-free variant of the p^T H p reduction, for callers that cannot allocate device
// memory themselves (a host application that owns the whole device-memory budget through its own allocator, such
// as a game engine or a renderer loading this library as a plugin, or a real-time thread that must never block
// in the driver's allocator).  The caller passes its own device buffers for the inputs and the output; the
// kernel's scratch (one partial sum per block and the arrival ticket of the last-block finish) lives in a
// file-scope __device__ array that every GPU loading the library holds until the process exits.
#include <mutex>
#include <string>

#include "../../include/pncg.h"
#include "common.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1 << 16;                                // 512 KiB of partial sums
constexpr long long NA_MAX_ITEMS = (long long)NA_THREADS * NA_MAX_BLOCKS;  // 16,777,216 tets or vertices
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    double partial[NA_MAX_BLOCKS];
    unsigned int ticket;
};

// The scratch: shared by every call on a device, it keeps the last call's contents.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoAllocScratch *g_scratch_ptr[NA_MAX_DEVICES] = {};
thread_local std::string g_noalloc_err;

// p^T M p + h^2 sum_e V_e [mu |dF|^2 + Psi_33 (cof F : dF)^2 + Psi_3 d2det(F)[dF, dF]] in double precision, one
// thread per tet (and per vertex for the inertia term); D_m^-1 and V_e are formed from the rest positions.
__global__ void __launch_bounds__(NA_THREADS) k_pHp_noalloc(NoAllocScratch *scr, int nv, int nt, const double *x,
                                                             const double *p, const double *X, const int *tets,
                                                             const double *mass, double mu, double lam, double h2,
                                                             double *out)
{
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s[1] = {0.0};
    if (i < nv) {
        const double px = p[3 * i], py = p[3 * i + 1], pz = p[3 * i + 2];
        s[0] += mass[i] * (px * px + py * py + pz * pz);
    }
    if (i < nt) {
        const int v[4] = {tets[4 * i], tets[4 * i + 1], tets[4 * i + 2], tets[4 * i + 3]};
        double A[3][3], Ds[3][3], Dp[3][3];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) {
                A[a][c] = X[3 * v[c + 1] + a] - X[3 * v[0] + a];
                Ds[a][c] = x[3 * v[c + 1] + a] - x[3 * v[0] + a];
                Dp[a][c] = p[3 * v[c + 1] + a] - p[3 * v[0] + a];
            }
        const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        double W[3][3];
        W[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
        W[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
        W[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
        W[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
        W[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
        W[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
        W[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
        W[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
        W[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
        double F[3][3], dF[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                F[a][b] = Ds[a][0] * W[0][b] + Ds[a][1] * W[1][b] + Ds[a][2] * W[2][b];
                dF[a][b] = Dp[a][0] * W[0][b] + Dp[a][1] * W[1][b] + Dp[a][2] * W[2][b];
            }
        // cofactor columns f1 x f2, f2 x f0, f0 x f1 of F and of the mixed terms
        double cf[3][3];
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            cf[0][b] = F[1][b1] * F[2][b2] - F[2][b1] * F[1][b2];
            cf[1][b] = F[2][b1] * F[0][b2] - F[0][b1] * F[2][b2];
            cf[2][b] = F[0][b1] * F[1][b2] - F[1][b1] * F[0][b2];
        }
        const double J = F[0][0] * cf[0][0] + F[1][0] * cf[1][0] + F[2][0] * cf[2][0];
        if (J > 0.0 && det > 0.0) {
            const double L = log(J);
            const double Psi3 = (lam * L - mu) / J, Psi33 = (mu + lam * (1.0 - L)) / (J * J);
            double n2 = 0.0, g3 = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) { n2 += dF[a][b] * dF[a][b]; g3 += cf[a][b] * dF[a][b]; }
            // d2det(F)[dF, dF] = 2 (df0 . (df1 x f2) + df0 . (f1 x df2) + f0 . (df1 x df2)), columns
            auto col = [](const double M[3][3], int b, double o[3]) { o[0] = M[0][b]; o[1] = M[1][b]; o[2] = M[2][b]; };
            auto tri = [](const double a[3], const double b[3], const double c[3]) {
                return a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
            };
            double f0[3], f1[3], f2[3], d0[3], d1[3], d2[3];
            col(F, 0, f0); col(F, 1, f1); col(F, 2, f2); col(dF, 0, d0); col(dF, 1, d1); col(dF, 2, d2);
            const double h3 = 2.0 * (tri(d0, d1, f2) + tri(d0, f1, d2) + tri(f0, d1, d2));
            s[0] += h2 * (det / 6.0) * (mu * n2 + Psi33 * g3 * g3 + Psi3 * h3);
        } else {
            s[0] = nan("");     // an inverted current tet, or a rest tet of non-positive volume
        }
    }
    pncg::block_sum<1>(s, sh);
    if (pncg::publish_partials<1>(s, scr->partial, &scr->ticket)) {
        double t[1];
        pncg::finish_sums<1>(t, scr->partial, sh);
        if (threadIdx.x == 0) *out = t[0];
    }
}

} // namespace

extern "C" {

const char *sim_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

sim_status sim_pHp_noalloc(int32_t n_verts, int32_t n_tets, const double *x, const double *p, const double *rest_x,
                           const int32_t *tets, const double *mass, double youngs, double poisson, double dt,
                           double *out, void *cuda_stream)
{
    if (n_verts <= 0 || n_tets <= 0 || !x || !p || !rest_x || !tets || !mass || !out || !(dt > 0) ||
        !(poisson > -1.0 && poisson < 0.5)) {
        g_noalloc_err = "sim_pHp_noalloc: invalid argument";
        return SIM_ERR_INVALID_ARG;
    }
    if ((long long)n_verts > NA_MAX_ITEMS || (long long)n_tets > NA_MAX_ITEMS) {
        g_noalloc_err = "sim_pHp_noalloc: at most " + std::to_string(NA_MAX_ITEMS) +
                        " tets and vertices per call (the static scratch holds " + std::to_string(NA_MAX_BLOCKS) +
                        " block partial sums)";
        return SIM_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        g_noalloc_err = "sim_pHp_noalloc: no usable CUDA device";
        return SIM_ERR_CUDA;
    }
    NoAllocScratch *scr;
    {
        // first call on this device: the scratch's device address (the symbol's host name is only a stand-in)
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                g_noalloc_err = std::string("sim_pHp_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
                return SIM_ERR_CUDA;
            }
            g_scratch_ptr[dev] = (NoAllocScratch *)ptr;
        }
        scr = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the arrival ticket must start at zero (the finishing block also resets it)
    e = cudaMemsetAsync(&scr->ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("sim_pHp_noalloc: ") + cudaGetErrorString(e);
        return SIM_ERR_CUDA;
    }
    const double mu = youngs / (2.0 * (1.0 + poisson)), lam = youngs * poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson));
    const int n = n_verts > n_tets ? n_verts : n_tets;
    const int blocks = (n + NA_THREADS - 1) / NA_THREADS;
    k_pHp_noalloc<<<blocks, NA_THREADS, 0, s>>>(scr, n_verts, n_tets, x, p, rest_x, tets, mass, mu, lam, dt * dt, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("sim_pHp_noalloc: launch failed: ") + cudaGetErrorString(e);
        return SIM_ERR_CUDA;
    }
    return SIM_OK;
}

} // extern "C"
