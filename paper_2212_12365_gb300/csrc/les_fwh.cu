// les_fwh: far-field acoustic pressure from the probe surface's frames by the
// Ffowcs Williams-Hawkings equation, the acoustic post-processing the paper's
// probe surface feeds (its Introduction and Concluding Remarks name FW-H for
// the far field but give no formulation).  Adopted formulation: Farassat's
// Formulation 1A (NASA TM-2007-214853) with the permeable-surface source
// terms of di Francescantonio (J. Sound Vib. 202, 1997), for a surface at rest
// in a medium at rest:
//     Q = rho u.n,   L_i = (p - p0) n_i + rho u_i u.n,
//     4 pi p'(x, t) = sum_panels A [ dQ/dtau / r + (dL_r/dtau) / (c0 r) + L_r / r^2 ]
// at the retarded time tau = t - r / c0, r = |x - y|, L_r = L.(x - y)/r.
// Discretisation: d/dtau by second-order central differences between frames
// (one-sided three-point at the first and last frame), retarded values by
// linear interpolation between the two frames around tau.
//
// Kernels.  k_fwh_src forms, per panel and frame, L and the derivatives
// dQ/dtau, dL/dtau in FP64 from the ring (either precision) and stores them as
// two float4 per (panel, frame), panel-major.  The observer pass, in one of
// two forms: k_fwh_obs_win (staged) takes a block of 256 observer times, a
// group of up to 16 microphones and a panel chunk per CTA, stages each
// panel's window of source frames in shared memory once and evaluates every
// microphone against it; k_fwh_obs (direct, when a window would not fit)
// takes one microphone per CTA and reads the frames from global memory.  In
// both, each thread is one observer time and sums its panels' contributions
// (compensated FP32 within a stage of panels, FP64 across stages), and each
// CTA writes its chunk's partial sums; k_fwh_sum adds the chunks in chunk
// order.  Every sum has a fixed order, so the result is the same on every run.
#include <cmath>
#include <string>
#include <vector>

#include "les_internal.cuh"

namespace les {

namespace {

constexpr int FWH_T = 256;   // observer times per CTA
constexpr int FWH_SUB = 256; // panels per shared-memory sub-chunk

// Ring frame m (0 = oldest used) of field f at panel j.
template <typename real>
__device__ __forceinline__ double ring_at(const real *ring, int first, int cap, int npts, int m, int f, int j)
{
    const int slot = (first + m) % cap;
    return (double)ring[((long long)slot * 5 + f) * npts + j];
}

// Q and L of panel j at ring frame m.
template <typename real>
__device__ __forceinline__ void ql_at(const real *ring, int first, int cap, int npts, int m, int j, const double n[3],
                                      double p0, double &Q, double L[3])
{
    const double rho = ring_at(ring, first, cap, npts, m, 0, j);
    const double u[3] = {ring_at(ring, first, cap, npts, m, 1, j), ring_at(ring, first, cap, npts, m, 2, j),
                         ring_at(ring, first, cap, npts, m, 3, j)};
    const double p = ring_at(ring, first, cap, npts, m, 4, j);
    const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    Q = rho * un;
    for (int i = 0; i < 3; ++i) L[i] = (p - p0) * n[i] + rho * u[i] * un;
}

// Per (panel j, frame m): src[(j*N + m)*2] = (L_x, L_y, L_z, dQ/dtau),
// src[(j*N + m)*2 + 1] = (dL_x/dtau, dL_y/dtau, dL_z/dtau, 0).  One thread per
// panel marches the frames with Q and L of three consecutive frames in
// registers, so each is formed once.
template <typename real>
__global__ void __launch_bounds__(256) k_fwh_src(const real *__restrict__ ring, int first, int cap, int npts, int N,
                                                 const double *__restrict__ nrm, double p0, double rdt2,
                                                 float4 *__restrict__ src)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npts) return;
    const double n[3] = {nrm[j], nrm[npts + j], nrm[2 * npts + j]};
    // Q and L of frames m-1 (a), m (b) and m+1 (c), shifted down each frame
    double Qa, La[3], Qb, Lb[3], Qc, Lc[3];
    ql_at(ring, first, cap, npts, 0, j, n, p0, Qa, La);
    ql_at(ring, first, cap, npts, 1, j, n, p0, Qb, Lb);
    ql_at(ring, first, cap, npts, 2, j, n, p0, Qc, Lc);
    float4 *o = src + (long long)j * N * 2;
    // first frame: one-sided three-point
    o[0] = make_float4((float)La[0], (float)La[1], (float)La[2], (float)((-3.0 * Qa + 4.0 * Qb - Qc) * rdt2));
    o[1] = make_float4((float)((-3.0 * La[0] + 4.0 * Lb[0] - Lc[0]) * rdt2),
                       (float)((-3.0 * La[1] + 4.0 * Lb[1] - Lc[1]) * rdt2),
                       (float)((-3.0 * La[2] + 4.0 * Lb[2] - Lc[2]) * rdt2), 0.0f);
    for (int m = 1; m < N - 1; ++m) {
        if (m > 1) { // frames m-1, m from the window, m+1 new
            Qa = Qb;
            Qb = Qc;
            for (int i = 0; i < 3; ++i) {
                La[i] = Lb[i];
                Lb[i] = Lc[i];
            }
            ql_at(ring, first, cap, npts, m + 1, j, n, p0, Qc, Lc);
        }
        o[2 * m] = make_float4((float)Lb[0], (float)Lb[1], (float)Lb[2], (float)((Qc - Qa) * rdt2));
        o[2 * m + 1] = make_float4((float)((Lc[0] - La[0]) * rdt2), (float)((Lc[1] - La[1]) * rdt2),
                                   (float)((Lc[2] - La[2]) * rdt2), 0.0f);
    }
    // last frame N - 1 (in c; N - 2 in b, N - 3 in a): one-sided three-point
    o[2 * (N - 1)] = make_float4((float)Lc[0], (float)Lc[1], (float)Lc[2], (float)((3.0 * Qc - 4.0 * Qb + Qa) * rdt2));
    o[2 * (N - 1) + 1] = make_float4((float)((3.0 * Lc[0] - 4.0 * Lb[0] + La[0]) * rdt2),
                                     (float)((3.0 * Lc[1] - 4.0 * Lb[1] + La[1]) * rdt2),
                                     (float)((3.0 * Lc[2] - 4.0 * Lb[2] + La[2]) * rdt2), 0.0f);
}

__global__ void __launch_bounds__(FWH_T) k_fwh_obs(const float4 *__restrict__ src, int npts, int N,
                                                   const double *__restrict__ xyz, const double *__restrict__ area,
                                                   const double *__restrict__ obs, int nobs, double t0, double dt_obs,
                                                   int nt, double dtau, double c0, int chunk,
                                                   double *__restrict__ part)
{
    __shared__ float4 geo[FWH_SUB]; // unit direction to the observer, A/(4 pi r)
    __shared__ float fr[FWH_SUB];   // fractional part of the panel's frame offset
    __shared__ float irs[FWH_SUB];  // 1/r
    __shared__ int mb[FWH_SUB];     // integer part of the panel's frame offset
    const int k = blockIdx.x * FWH_T + threadIdx.x;
    const int o = blockIdx.y, c = blockIdx.z;
    const double ox = obs[o], oy = obs[nobs + o], oz = obs[2 * nobs + o];
    // The emission time of observer time t_k at distance r, in frames, is
    // s = t_k / dtau - r / (c0 dtau).  Split exactly in FP64 into a CTA base B
    // (an integer), the thread's small offset t_k/dtau - B (FP32) and the
    // panel's offset B - r/(c0 dtau) = M + f (integer M, fraction f in FP32),
    // so that the per-panel work of a thread is FP32 and integer arithmetic.
    const double B = floor((t0 + (double)(blockIdx.x * FWH_T) * dt_obs) / dtau);
    const float skl = (float)((t0 + (double)k * dt_obs) / dtau - B);
    const float rc0 = (float)(1.0 / c0);
    const int j0 = c * chunk, j1 = min(npts, j0 + chunk);
    double acc = 0.0;
    for (int jb = j0; jb < j1; jb += FWH_SUB) {
        const int nsub = min(FWH_SUB, j1 - jb);
        __syncthreads(); // the previous sub-chunk's geometry is no longer read
        if (threadIdx.x < nsub) {
            const int j = jb + threadIdx.x;
            const double dx = ox - xyz[j], dy = oy - xyz[npts + j], dz = oz - xyz[2 * npts + j];
            const double r = sqrt(dx * dx + dy * dy + dz * dz), ir = 1.0 / r;
            geo[threadIdx.x] = make_float4((float)(dx * ir), (float)(dy * ir), (float)(dz * ir),
                                           (float)(area[j] * ir / (4.0 * M_PI)));
            const double e = B - r / (c0 * dtau);
            const double ef = floor(e);
            mb[threadIdx.x] = (int)ef;
            fr[threadIdx.x] = (float)(e - ef);
            irs[threadIdx.x] = (float)ir;
        }
        __syncthreads();
        if (k < nt) {
            float sum = 0.0f, comp = 0.0f; // compensated sum over the sub-chunk
            for (int q = 0; q < nsub; ++q) {
                const float4 g = geo[q];
                const float s = skl + fr[q];
                const float fl = floorf(s);
                int m = mb[q] + (int)fl;
                m = m < 0 ? 0 : (m > N - 2 ? N - 2 : m);
                const float w = s - fl;
                const float4 *p = src + ((long long)(jb + q) * N + m) * 2;
                const float4 a0 = p[0], b0 = p[1], a1 = p[2], b1 = p[3];
                const float Lx = fmaf(w, a1.x - a0.x, a0.x), Ly = fmaf(w, a1.y - a0.y, a0.y),
                            Lz = fmaf(w, a1.z - a0.z, a0.z), dQ = fmaf(w, a1.w - a0.w, a0.w);
                const float dLx = fmaf(w, b1.x - b0.x, b0.x), dLy = fmaf(w, b1.y - b0.y, b0.y),
                            dLz = fmaf(w, b1.z - b0.z, b0.z);
                const float Lr = fmaf(Lx, g.x, fmaf(Ly, g.y, Lz * g.z));
                const float dLr = fmaf(dLx, g.x, fmaf(dLy, g.y, dLz * g.z));
                // A/(4 pi r) [dQ + dL_r / c0 + L_r / r]
                const float v = g.w * fmaf(Lr, irs[q], fmaf(dLr, rc0, dQ));
                const float y = v - comp;
                const float tsum = sum + y;
                comp = (tsum - sum) - y;
                sum = tsum;
            }
            acc += (double)sum;
        }
    }
    if (k < nt) part[((long long)c * nobs + o) * nt + k] = acc;
}

// Observer pass with shared-memory reuse: a CTA per (256 observer times,
// group of up to MG microphones, panel chunk).  Per group of G panels the CTA
// forms every (panel, microphone) geometry, stages each panel's window of W
// consecutive source frames (all the emission frames any of its microphones
// needs for the block's 256 times) from global into shared memory once, and
// then every thread (one observer time) evaluates all microphones against the
// staged windows, with a compensated FP32 sum over the group's panels added
// to its FP64 accumulator per microphone (in shared memory).  Each source
// frame is read from global memory once per CTA instead of once per
// (microphone, time) evaluation.
__global__ void __launch_bounds__(FWH_T) k_fwh_obs_win(const float4 *__restrict__ src, int npts, int N,
                                                       const double *__restrict__ xyz, const double *__restrict__ area,
                                                       const double *__restrict__ obs, int nobs, int MG, double t0,
                                                       double dt_obs, int nt, double dtau, double c0, int chunk, int G,
                                                       int W, double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char fwh_sm[];
    const int o0 = blockIdx.y * MG, mgt = min(MG, nobs - o0);
    double *acc = (double *)fwh_sm;                           // [MG][FWH_T]
    float4 *geo = (float4 *)(acc + (size_t)MG * FWH_T);       // [G][MG][2]
    float4 *winA = geo + (size_t)G * MG * 2;                  // [G][W]: (L, dQ/dtau)
    float4 *winB = winA + (size_t)G * W;                      // [G][W]: dL/dtau (16-byte lane stride)
    int *mlo = (int *)(winB + (size_t)G * W);                 // [G]
    const int tid = threadIdx.x;
    const int k = blockIdx.x * FWH_T + tid;
    const int c = blockIdx.z;
    const double B = floor((t0 + (double)(blockIdx.x * FWH_T) * dt_obs) / dtau);
    const float skl = (float)((t0 + (double)k * dt_obs) / dtau - B);
    const float rc0 = (float)(1.0 / c0);
    for (int o = 0; o < mgt; ++o) acc[o * FWH_T + tid] = 0.0;
    const int j0 = c * chunk, j1 = min(npts, j0 + chunk);
    for (int jb = j0; jb < j1; jb += G) {
        const int ng = min(G, j1 - jb);
        __syncthreads(); // the previous group's geometry and windows are no longer read
        for (int i = tid; i < ng * mgt; i += FWH_T) {
            const int g = i / mgt, o = i - g * mgt, j = jb + g;
            const double dx = obs[o0 + o] - xyz[j], dy = obs[nobs + o0 + o] - xyz[npts + j],
                         dz = obs[2 * nobs + o0 + o] - xyz[2 * npts + j];
            const double r = sqrt(dx * dx + dy * dy + dz * dz), ir = 1.0 / r;
            const double e = B - r / (c0 * dtau);
            const double ef = floor(e);
            geo[(g * MG + o) * 2] = make_float4((float)(dx * ir), (float)(dy * ir), (float)(dz * ir),
                                                (float)(area[j] * ir / (4.0 * M_PI)));
            geo[(g * MG + o) * 2 + 1] = make_float4((float)(e - ef), __int_as_float((int)ef), (float)ir, 0.0f);
        }
        __syncthreads();
        if (tid < ng) { // window start: the earliest frame any microphone needs
            int m = 0x7fffffff;
            for (int o = 0; o < mgt; ++o) m = min(m, __float_as_int(geo[(tid * MG + o) * 2 + 1].y));
            mlo[tid] = max(m, 0);
        }
        __syncthreads();
        for (int i = tid; i < ng * W * 2; i += FWH_T) {
            const int g = i / (2 * W), r2 = i - g * 2 * W;
            const int f = min(mlo[g] + (r2 >> 1), N - 1);
            (r2 & 1 ? winB : winA)[g * W + (r2 >> 1)] = src[((long long)(jb + g) * N + f) * 2 + (r2 & 1)];
        }
        __syncthreads();
        if (k < nt) {
            for (int o = 0; o < mgt; ++o) {
                float sum = 0.0f, comp = 0.0f;
                for (int g = 0; g < ng; ++g) {
                    const float4 gd = geo[(g * MG + o) * 2], h = geo[(g * MG + o) * 2 + 1];
                    const float s = skl + h.x;
                    const float fl = floorf(s);
                    int m = __float_as_int(h.y) + (int)fl;
                    m = m < 0 ? 0 : (m > N - 2 ? N - 2 : m);
                    int idx = m - mlo[g];
                    idx = idx < 0 ? 0 : (idx > W - 2 ? W - 2 : idx);
                    const float w = s - fl;
                    const float4 *pa = winA + g * W + idx, *pb = winB + g * W + idx;
                    const float4 a0 = pa[0], a1 = pa[1], b0 = pb[0], b1 = pb[1];
                    const float Lx = fmaf(w, a1.x - a0.x, a0.x), Ly = fmaf(w, a1.y - a0.y, a0.y),
                                Lz = fmaf(w, a1.z - a0.z, a0.z), dQ = fmaf(w, a1.w - a0.w, a0.w);
                    const float dLx = fmaf(w, b1.x - b0.x, b0.x), dLy = fmaf(w, b1.y - b0.y, b0.y),
                                dLz = fmaf(w, b1.z - b0.z, b0.z);
                    const float Lr = fmaf(Lx, gd.x, fmaf(Ly, gd.y, Lz * gd.z));
                    const float dLr = fmaf(dLx, gd.x, fmaf(dLy, gd.y, dLz * gd.z));
                    const float v = gd.w * fmaf(Lr, h.z, fmaf(dLr, rc0, dQ));
                    const float y = v - comp;
                    const float tsum = sum + y;
                    comp = (tsum - sum) - y;
                    sum = tsum;
                }
                acc[o * FWH_T + tid] += (double)sum;
            }
        }
    }
    if (k < nt)
        for (int o = 0; o < mgt; ++o) part[((long long)c * nobs + o0 + o) * nt + k] = acc[o * FWH_T + tid];
}

__global__ void k_fwh_sum(const double *__restrict__ part, int nchunk, long long n, double *__restrict__ out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * n + i];
    out[i] = s;
}

} // namespace

} // namespace les

using namespace les;

extern "C" int les_fwh(const void *ring, int precision, int capacity, int64_t frames_written, int npts,
                       const double *xyz, const double *nrm, const double *area, double dtau, double p0, double c0,
                       int nobs, const double *obs, double t0, double dt_obs, int nt, double *p_out, void *stream,
                       double *ms_out)
{
    auto bad = [](const char *msg) {
        set_call_error(msg);
        return LES_ERR_ARG;
    };
    set_call_error("");
    if (!ring || !xyz || !nrm || !area || !obs || !p_out) return bad("null pointer");
    if (precision != LES_FP64 && precision != LES_FP32 && precision != LES_FP32_SEPARABLE)
        return bad("unknown precision");
    if (npts < 1 || nobs < 1 || nt < 1 || capacity < 1) return bad("npts, nobs, nt and capacity must be >= 1");
    const int N = (int)std::min<int64_t>(frames_written, capacity);
    if (frames_written < 3 || N < 3) return bad("at least three frames are needed");
    if (!(dtau > 0) || !(c0 > 0) || !(dt_obs >= 0)) return bad("dtau and c0 must be > 0, dt_obs >= 0");
    // every emission time of every panel must lie within the frames; on the
    // way, the largest spread of a panel's distances over a group of 16
    // microphones (the window the staged observer pass needs)
    const double tau_max = (N - 1) * dtau, t1 = t0 + (nt - 1) * dt_obs;
    std::vector<double> gmin((size_t)npts), gmax((size_t)npts);
    double spread16 = 0.0;
    for (int o = 0; o < nobs; ++o) {
        double rmin = 1e300, rmax = 0.0;
        const bool g0 = o % 16 == 0;
        for (int j = 0; j < npts; ++j) {
            const double dx = obs[o] - xyz[j], dy = obs[nobs + o] - xyz[npts + j], dz = obs[2 * nobs + o] - xyz[2 * npts + j];
            const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r > 0)) return bad("an observer coincides with a panel");
            rmin = std::min(rmin, r);
            rmax = std::max(rmax, r);
            gmin[j] = g0 ? r : std::min(gmin[j], r);
            gmax[j] = g0 ? r : std::max(gmax[j], r);
        }
        if (o % 16 == 15 || o == nobs - 1)
            for (int j = 0; j < npts; ++j) spread16 = std::max(spread16, gmax[j] - gmin[j]);
        if (t0 - rmax / c0 < 0.0 || t1 - rmin / c0 > tau_max)
            return bad("an emission time t - r/c0 falls outside the frames: need t0 >= r_max/c0 and "
                       "t0 + (nt-1) dt_obs - r_min/c0 <= (frames - 1) dtau");
    }
    const int first = (int)((frames_written - N) % capacity);
    cudaStream_t st = (cudaStream_t)stream;
    // panel-chunk count: about four CTAs per SM in total
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LES_ERR_CUDA;
    const int tblocks = (nt + FWH_T - 1) / FWH_T;
    // The staged observer pass (k_fwh_obs_win) with microphone groups of 16:
    // a window of W frames per panel (the block's 256 times plus the spread of
    // the group's emission times), G panels per stage within ~100 KB of shared
    // memory; if fewer than 4 panels fit, the direct pass (k_fwh_obs).
    const int MG = std::min(16, nobs), ngroups = (nobs + MG - 1) / MG;
    const double W_d = std::ceil(spread16 / (c0 * dtau)) + std::ceil((FWH_T - 1) * dt_obs / dtau) + 4.0;
    const int W = W_d < 1e6 ? (int)W_d : 1000000;
    const size_t budget = 100 * 1024, acc_b = (size_t)MG * FWH_T * 8; // two CTAs per SM
    const int G = (int)std::min<size_t>(32, (budget - acc_b) / (32 * ((size_t)MG + W) + 4));
    const bool staged = G >= 4;
    const size_t win_smem = acc_b + (size_t)G * MG * 32 + (size_t)G * W * 32 + (size_t)G * 4;
    int nchunk, chunk;
    if (staged) {
        nchunk = std::max(1, std::min(npts, (2 * nsm + tblocks * ngroups - 1) / (tblocks * ngroups)));
        chunk = (npts + nchunk - 1) / nchunk;
        nchunk = (npts + chunk - 1) / chunk;
        if (cudaFuncSetAttribute(k_fwh_obs_win, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem) !=
            cudaSuccess)
            return LES_ERR_CUDA;
    } else {
        nchunk = (4 * nsm + tblocks * nobs - 1) / (tblocks * nobs);
        nchunk = std::max(1, std::min(nchunk, (npts + FWH_SUB - 1) / FWH_SUB));
        chunk = ((npts + nchunk - 1) / nchunk + FWH_SUB - 1) / FWH_SUB * FWH_SUB;
        nchunk = (npts + chunk - 1) / chunk;
    }
    const size_t n_src = (size_t)npts * N * 2;
    const size_t n_out = (size_t)nobs * nt;
    float4 *d_src = nullptr;
    double *d_geo = nullptr, *d_part = nullptr;
    const size_t geo_doubles = (size_t)npts * 7 + (size_t)nobs * 3;
    auto release = [&]() {
        if (d_src) cudaFree(d_src);
        if (d_geo) cudaFree(d_geo);
        if (d_part) cudaFree(d_part);
    };
    if (cudaMalloc(&d_src, n_src * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&d_geo, geo_doubles * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_part, (n_out * (nchunk + 1)) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        release();
        set_call_error("device allocation failed");
        return LES_ERR_OOM;
    }
    double *d_xyz = d_geo, *d_nrm = d_geo + 3 * (size_t)npts, *d_area = d_geo + 6 * (size_t)npts,
           *d_obs = d_geo + 7 * (size_t)npts, *d_out = d_part + n_out * nchunk;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int rc = LES_OK;
    if (cudaMemcpyAsync(d_xyz, xyz, 3 * (size_t)npts * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_nrm, nrm, 3 * (size_t)npts * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_area, area, (size_t)npts * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_obs, obs, 3 * (size_t)nobs * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = LES_ERR_CUDA;
    if (rc == LES_OK && ms_out)
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) rc = LES_ERR_CUDA;
    if (rc == LES_OK) {
        if (ms_out) cudaEventRecord(ev[0], st);
        const int grid = (npts + 255) / 256;
        const double rdt2 = 1.0 / (2.0 * dtau);
        if (precision == LES_FP64)
            k_fwh_src<double><<<grid, 256, 0, st>>>((const double *)ring, first, capacity, npts, N, d_nrm, p0, rdt2, d_src);
        else
            k_fwh_src<float><<<grid, 256, 0, st>>>((const float *)ring, first, capacity, npts, N, d_nrm, p0, rdt2, d_src);
        if (ms_out) cudaEventRecord(ev[1], st);
        if (staged)
            k_fwh_obs_win<<<dim3(tblocks, ngroups, nchunk), FWH_T, win_smem, st>>>(
                d_src, npts, N, d_xyz, d_area, d_obs, nobs, MG, t0, dt_obs, nt, dtau, c0, chunk, G, W, d_part);
        else
            k_fwh_obs<<<dim3(tblocks, nobs, nchunk), FWH_T, 0, st>>>(d_src, npts, N, d_xyz, d_area, d_obs, nobs, t0,
                                                                     dt_obs, nt, dtau, c0, chunk, d_part);
        if (ms_out) cudaEventRecord(ev[2], st);
        k_fwh_sum<<<(int)((n_out + 255) / 256), 256, 0, st>>>(d_part, nchunk, (long long)n_out, d_out);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(p_out, d_out, n_out * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = LES_ERR_CUDA;
        if (rc == LES_OK && ms_out) {
            float a = 0.0f, b = 0.0f;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b, ev[1], ev[2]);
            ms_out[0] = a;
            ms_out[1] = b;
        }
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (rc != LES_OK) {
        cudaGetLastError();
        set_call_error("CUDA failure in the FW-H evaluation");
    }
    release();
    return rc;
}
