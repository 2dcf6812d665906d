// Setup kernels: element geometry of the linear triangles and the constant
// matrices of the semi-discrete eddy-current system (Sec. 2, Eq. 1):
//   K_lin,ab = sum_e nu_e |e| grad N_a . grad N_b     (linear materials)
//   M_ab     = sum_e sigma_e |e| (1 + delta_ab) / 12   (conductive regions)
//   g_a      = sum_{e in source, a in e} |e| / 3 / A_source
// plus the tables used by the per-lane nonlinear assembly and the DFT
// twiddles exp(-i 2 pi k / N) of the multi-harmonic coarse solve (Eqs. 11-13).
// K_lin u is evaluated in the kernels in the difference form
//   (K_lin u)_i = sum_{j != i} K_ij (u_j - u_i) + dlin_i u_i,
// dlin_i = sum_j K_ij (free columns), which keeps the rounding error of the
// residual proportional to the differences of u rather than to u itself.
// Every entry is a gather over the element contributions listed for it on the
// host, so no atomics are used and the results are deterministic.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace pppc {
namespace {

constexpr int kMatStride = 8;  // sigma, nu_model, nu, k1, k2, k3, is_source, cap on |B|^2

__global__ void geom_kernel(SetupArgs a) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.n_tri; e += gridDim.x * blockDim.x) {
        const int v0 = a.tri[3 * e], v1 = a.tri[3 * e + 1], v2 = a.tri[3 * e + 2];
        const double x0 = a.xy[2 * v0], y0 = a.xy[2 * v0 + 1];
        const double x1 = a.xy[2 * v1], y1 = a.xy[2 * v1 + 1];
        const double x2 = a.xy[2 * v2], y2 = a.xy[2 * v2 + 1];
        const double det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        double* G = a.geom + 8 * (size_t)e;
        if (!(det != 0.0) || !isfinite(det)) {
            set_status(a.status, DEV_ERR_GEOMETRY);
            for (int q = 0; q < 8; ++q) G[q] = 0.0;
            continue;
        }
        G[0] = 0.5 * fabs(det);
        G[1] = (y1 - y2) / det;
        G[2] = (x2 - x1) / det;
        G[3] = (y2 - y0) / det;
        G[4] = (x0 - x2) / det;
        G[5] = (y0 - y1) / det;
        G[6] = (x1 - x0) / det;
        G[7] = 0.0;
    }
}

__device__ __forceinline__ double gdot(const double* G, int a, int b) {
    return G[1 + 2 * a] * G[1 + 2 * b] + G[2 + 2 * a] * G[2 + 2 * b];
}

// K_lin per row; invdiag_lin from its diagonal (non-special rows use it).
__global__ void klin_kernel(SetupArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.ndof; i += gridDim.x * blockDim.x) {
        for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
            double v = 0.0;
            for (int c = a.contrib_ptr[k]; c < a.contrib_ptr[k + 1]; ++c) {
                const int pk = a.contrib[c];
                const int e = pk / 9, ab = pk % 9;
                const double* m = a.mat + kMatStride * a.region[e];
                if (m[1] != 0.0) continue;  // nonlinear material: assembled per lane
                const double* G = a.geom + 8 * (size_t)e;
                v += m[2] * G[0] * gdot(G, ab / 3, ab % 3);
            }
            a.Klin[k] = v;
            a.Klin32[k] = (float)v;
        }
        // Row sum of K_lin over the free columns.  Each element's rows sum to
        // zero (sum_b grad N_b = 0), so it equals minus the couplings to the
        // eliminated Dirichlet nodes: exactly zero away from the boundary.
        double dsum = 0.0;
        for (int c = a.dcoup_ptr[i]; c < a.dcoup_ptr[i + 1]; ++c) {
            const int pk = a.dcoup[c];
            const int e = pk / 9, ab = pk % 9;
            const double* m = a.mat + kMatStride * a.region[e];
            if (m[1] != 0.0) continue;
            const double* G = a.geom + 8 * (size_t)e;
            dsum -= m[2] * G[0] * gdot(G, ab / 3, ab % 3);
        }
        a.dlin[i] = dsum;
        const double dg = a.Klin[a.diag_k[i]];
        a.invdiag_lin[i] = dg != 0.0 ? 1.0 / dg : 0.0;
        a.invdiag_lin32[i] = (float)a.invdiag_lin[i];
    }
}

__global__ void mass_kernel(SetupArgs a) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.n_slots; s += gridDim.x * blockDim.x) {
        const int k = a.slot_k[s];
        double v = 0.0;
        for (int c = a.contrib_ptr[k]; c < a.contrib_ptr[k + 1]; ++c) {
            const int pk = a.contrib[c];
            const int e = pk / 9, ab = pk % 9;
            const double sigma = a.mat[kMatStride * a.region[e]];
            if (sigma > 0.0) v += sigma * a.geom[8 * (size_t)e] * ((ab / 3 == ab % 3) ? 2.0 : 1.0) / 12.0;
        }
        a.Mslot[s] = v;
    }
}

// Single-block fixed-order sum of the source-element areas.
__global__ void source_area_kernel(SetupArgs a) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int e = threadIdx.x; e < a.n_tri; e += blockDim.x)
        if (a.mat[kMatStride * a.region[e] + 6] != 0.0) acc += a.geom[8 * (size_t)e];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.scalars[0] = red[0];
}

__global__ void source_shape_kernel(SetupArgs a) {
    const double area = a.scalars[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.ndof; i += gridDim.x * blockDim.x) {
        const int k = a.diag_k[i];
        double v = 0.0;
        for (int c = a.contrib_ptr[k]; c < a.contrib_ptr[k + 1]; ++c) {
            const int e = a.contrib[c] / 9;
            if (a.mat[kMatStride * a.region[e] + 6] != 0.0) v += a.geom[8 * (size_t)e] / 3.0;
        }
        a.g[i] = area > 0.0 ? v / area : 0.0;
    }
}

__global__ void norm_g_kernel(SetupArgs a) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < a.ndof; i += blockDim.x) acc += a.g[i] * a.g[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.scalars[1] = sqrt(red[0]);
}

__global__ void nl_tables_kernel(SetupArgs a) {
    const int stride = gridDim.x * blockDim.x;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n_nl; q += stride) {
        const int e = a.nl_elems[q];
        for (int t = 0; t < 8; ++t) a.nl_geom[8 * (size_t)q + t] = a.geom[8 * (size_t)e + t];
        const double* m = a.mat + kMatStride * a.region[e];
        a.nl_k[4 * (size_t)q + 0] = m[3];
        a.nl_k[4 * (size_t)q + 1] = m[4];
        a.nl_k[4 * (size_t)q + 2] = m[5];
        a.nl_k[4 * (size_t)q + 3] = m[7];
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.n_nlc; c += stride) {
        const int pk = a.nlc[c];
        const int e = a.nl_elems[pk / 9], ab = pk % 9;
        a.nlc_ab[c] = gdot(a.geom + 8 * (size_t)e, ab / 3, ab % 3);
    }
}

__global__ void twiddle_kernel(SetupArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.N; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)a.N, &s, &c);
        a.tw[2 * k] = c;
        a.tw[2 * k + 1] = -s;
    }
}

inline int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535) b = 65535;
    return (int)b;
}

}  // namespace

cudaError_t launch_setup(const SetupArgs& a, cudaStream_t st) {
    geom_kernel<<<grid_for(a.n_tri, 256), 256, 0, st>>>(a);
    klin_kernel<<<grid_for(a.ndof, 256), 256, 0, st>>>(a);
    if (a.n_slots > 0) mass_kernel<<<grid_for(a.n_slots, 256), 256, 0, st>>>(a);
    source_area_kernel<<<1, 256, 0, st>>>(a);
    source_shape_kernel<<<grid_for(a.ndof, 256), 256, 0, st>>>(a);
    norm_g_kernel<<<1, 256, 0, st>>>(a);
    if (a.n_nl > 0 || a.n_nlc > 0)
        nl_tables_kernel<<<grid_for(a.n_nl > a.n_nlc ? a.n_nl : a.n_nlc, 256), 256, 0, st>>>(a);
    twiddle_kernel<<<grid_for(a.N, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pppc
