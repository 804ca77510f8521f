// les_diag_sums_noalloc: the residual / conservation reduction of
// les_get_diagnostics for callers that must not allocate device memory.
//
// Who needs it: code that runs inside a framework whose caching allocator has
// reserved (nearly) all device memory, so a cudaMalloc would fail or fragment
// the pool; and monitoring hooks called every step, where cudaMalloc/cudaFree
// would add allocation latency and may synchronise the whole device, stalling
// other streams.  Such callers pass their own state and residual buffers and
// get the sums back in their own output buffer; this entry point allocates
// nothing (no cudaMalloc, cudaFree or allocating library call).
//
// Its only scratch is the file-scope array g_partials below: one slot of
// NA_NPART doubles per reduction block, at most NA_MAX_BLOCKS blocks.  Every
// GPU that loads the library holds it (557 KB) until the process exits.
#include <cstdio>
#include <mutex>

#include "les_internal.cuh"

namespace {

constexpr int NA_BLOCK = 256;                      // threads per reduction block
constexpr long long NA_POINTS_PER_BLOCK = 65536;   // points summed by one block
constexpr int NA_MAX_BLOCKS = LES_NOALLOC_MAX_POINTS / 65536;
constexpr int NA_NPART = 17;                       // partial results per block
static_assert((long long)NA_MAX_BLOCKS * NA_POINTS_PER_BLOCK == LES_NOALLOC_MAX_POINTS,
              "scratch size and the documented limit must agree");

// Per-block partials: [0] max|RHS_rho|, [1..5] sum RHS_f^2, [6..10] Neumaier
// sums of Qhat_f, [11..15] their compensations, [16] non-finite count.  Every
// call overwrites the slots of the blocks it launches; nothing needs clearing.
static __device__ __align__(256) double g_partials[NA_MAX_BLOCKS * NA_NPART];

__device__ __forceinline__ void na_neumaier(double &s, double &c, double v)
{
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// Block b sums points [b*NA_POINTS_PER_BLOCK, (b+1)*NA_POINTS_PER_BLOCK) in a
// fixed order (thread stride, then a shared-memory tree), so the result
// depends only on the inputs and npoints.
__global__ void __launch_bounds__(NA_BLOCK) k_na_partials(const double *__restrict__ qhat,
                                                          const double *__restrict__ rhs,
                                                          long long npoints, double *part)
{
    __shared__ double sh[NA_NPART][NA_BLOCK];
    const long long p0 = (long long)blockIdx.x * NA_POINTS_PER_BLOCK;
    long long p1 = p0 + NA_POINTS_PER_BLOCK;
    if (p1 > npoints) p1 = npoints;
    double mx = 0.0, bad = 0.0, l2[5] = {0, 0, 0, 0, 0}, s[5] = {0, 0, 0, 0, 0},
           c[5] = {0, 0, 0, 0, 0};
    for (long long p = p0 + threadIdx.x; p < p1; p += NA_BLOCK) {
        for (int f = 0; f < 5; ++f) {
            double r = rhs[f * npoints + p];
            double v = qhat[f * npoints + p];
            if (!isfinite(r) || !isfinite(v)) bad += 1.0;
            l2[f] += r * r;
            na_neumaier(s[f], c[f], v);
        }
        mx = fmax(mx, fabs(rhs[p]));
    }
    sh[0][threadIdx.x] = mx;
    for (int f = 0; f < 5; ++f) {
        sh[1 + f][threadIdx.x] = l2[f];
        sh[6 + f][threadIdx.x] = s[f];
        sh[11 + f][threadIdx.x] = c[f];
    }
    sh[16][threadIdx.x] = bad;
    __syncthreads();
    for (int st = NA_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            const int o = threadIdx.x + st;
            sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][o]);
            for (int f = 0; f < 5; ++f) {
                sh[1 + f][threadIdx.x] += sh[1 + f][o];
                double a = sh[6 + f][threadIdx.x], ca = sh[11 + f][threadIdx.x];
                na_neumaier(a, ca, sh[6 + f][o]);
                sh[6 + f][threadIdx.x] = a;
                sh[11 + f][threadIdx.x] = ca + sh[11 + f][o];
            }
            sh[16][threadIdx.x] += sh[16][o];
        }
        __syncthreads();
    }
    if (threadIdx.x < NA_NPART) part[blockIdx.x * NA_NPART + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_na_final(const double *__restrict__ part, int nblocks, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mx = 0.0, bad = 0.0, l2[5] = {0, 0, 0, 0, 0}, s[5] = {0, 0, 0, 0, 0},
           c[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b) {
        const double *P = part + (long long)b * NA_NPART;
        mx = fmax(mx, P[0]);
        for (int f = 0; f < 5; ++f) {
            l2[f] += P[1 + f];
            na_neumaier(s[f], c[f], P[6 + f]);
            c[f] += P[11 + f];
        }
        bad += P[16];
    }
    out[0] = mx;
    for (int f = 0; f < 5; ++f) {
        out[1 + f] = sqrt(l2[f]);
        out[6 + f] = s[f] + c[f];
    }
    out[11] = bad;
}

// Device address of g_partials per device.  In host code the name
// g_partials denotes a host-side stand-in, not device memory, so the address
// is looked up once per device (with that device current) and cached.
constexpr int NA_MAX_DEVICES = 64;
double *g_partials_addr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_setup_mutex;

} // namespace

extern "C" int les_diag_sums_noalloc(const double *qhat, const double *rhs, int64_t npoints,
                                     double *out, void *stream)
{
    if (!qhat || !rhs || !out || npoints < 1) return LES_ERR_ARG;
    if (npoints > (int64_t)LES_NOALLOC_MAX_POINTS) {
        std::fprintf(stderr,
                     "les_diag_sums_noalloc: %lld points exceed the fixed scratch limit of %lld "
                     "points; use les_get_diagnostics for larger grids\n",
                     (long long)npoints, (long long)LES_NOALLOC_MAX_POINTS);
        return LES_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LES_ERR_CUDA;
    double *part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return LES_ERR_CUDA;
            }
            g_partials_addr[dev] = (double *)p;
        }
        part = g_partials_addr[dev];
    }
    const int nblocks = (int)((npoints + NA_POINTS_PER_BLOCK - 1) / NA_POINTS_PER_BLOCK);
    cudaStream_t st = (cudaStream_t)stream;
    k_na_partials<<<nblocks, NA_BLOCK, 0, st>>>(qhat, rhs, (long long)npoints, part);
    k_na_final<<<1, 32, 0, st>>>(part, nblocks, out);
    if (cudaGetLastError() != cudaSuccess) return LES_ERR_CUDA;
    return LES_OK;
}
