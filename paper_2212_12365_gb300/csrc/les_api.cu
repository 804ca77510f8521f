// Host runtime of libles.so: handles, device memory plan, CUDA-graph step,
// state transfer, diagnostics and the surface probe behind the C ABI of les.h.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "les_internal.cuh"

using namespace les;

namespace {

// Host record of one jet: dimensions, parameters, device pointers.
struct JetHost {
    int n[3];
    int pitch;
    long long fs;
    long long npad;
    long long N;
    int per[3];
    int bc[6];
    double shift[9];
    les_params prm;
    bool product;                      // Cartesian-product grid (probe support)
    std::vector<double> ax[3];         // 1-D coordinates of a product grid
    size_t off;                        // byte offset of this jet's region
    size_t bytes;                      // size of this jet's region
    // device pointers (typed as bytes; the element type follows the precision)
    char *met, *q[3], *prim, *grad, *hflux, *rhs;
    double *jinv64, *inflow_ut;
    float4 *h1[3];                     // FP32: 1-D spacings of a product grid (separable form)
    float4 *mp;                        // FP32 general form: paired static records (5 float4 / row pair)
    int nblk_pt, nblk_bc[3];
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr int DIAG_BLOCKS = 608; // blocks of the diagnostics reduction (fixed order)

} // namespace

struct les_handle {
    int prec = LES_FP64;        // LES_FP64 or LES_FP32 (storage and arithmetic)
    bool sep = false;           // FP32 separable-metric stage (LES_FP32_SEPARABLE)
    bool centerline = false;    // some jet has a centerline face
    int max_ni = 0;
    int njets = 0;
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;
    int nsm = 152;
    int dev = 0;
    char *base = nullptr;
    size_t bytes = 0;
    bool owns = false;
    std::vector<JetHost> J;
    void *d_jets = nullptr;     // JetDev<real>[njets]
    int *d_maps = nullptr;      // block-start tables
    BlockMap pt{}, bcm[3]{};
    std::vector<BlockMap> pt1, bc1[3]; // single-jet maps
    double *d_dt = nullptr;
    long long *d_level = nullptr;
    unsigned long long *d_dtbits = nullptr;
    double *d_partials = nullptr;
    double *d_diag = nullptr;
    long long *d_probe_base = nullptr;
    double *d_stage = nullptr;   // 5*max(N) doubles: host transfer staging
    // error word: the first out-of-range index (bounds-checked builds) or a
    // staging wait of the fused stage that gave up (site 8, every build)
    unsigned long long *d_oob = nullptr;
    int stage_wait_limit = -1; // polls per staging wait of the fused stage (-1: the default)
    CUtensorMap *d_tmap = nullptr; // per jet: TMA maps of the 3 state registers for TY 8 and 16
    int nblk_diag = 0;
    int64_t step = 0;
    std::vector<double> dt;
    std::vector<char> has_state;
    cudaGraphExec_t gexec = nullptr;
    // fused FP32 stage: work-list tables (all jets; and one per jet with item0 = 0)
    FusedJet *d_fj = nullptr, *d_fj1 = nullptr;
    std::vector<FusedJet> fj, fj1; // host copies of d_fj and d_fj1
    std::vector<JetDev<float>> jd32; // host copy of the FP32 jet table
    int fused_ty = 16;
    int fused_balanced = 0; // 0: k-chunk items, 1: balanced ranges, 2: lockstep waves, then balanced ranges
    int fused_items = 0, fused_tiles = 0;
    int fused_cps[2] = {1, 1}; // resident CTAs per SM of the fused stage at tile height 8, 16
    bool tuned = false;
    std::string tune_note;
    int64_t launches_per_step = 0;
    int64_t last_launches = 0;
    // probe
    int probe_npts = 0, probe_every = 1, probe_cap = 0;
    int64_t probe_base_level = 0;
    void *probe_out = nullptr;
    int *d_cell = nullptr;
    double *d_wts = nullptr;
    std::string err;
};

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                           \
            return LES_ERR_CUDA;                                                                   \
        }                                                                                          \
    } while (0)

// Text of the last failed les_create_grid / les_create_batch of this thread
// (returned by les_last_error(NULL)).
static thread_local std::string g_create_err;

namespace les {
void set_call_error(const char *msg) { g_create_err = msg; }
} // namespace les

static int fail(les_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

// Status of the fused FP32 stage's bounded staging waits (call after a stream
// synchronisation): LES_ERR_TIMEOUT once a wait has given up (site 8 in the
// handle's error word; the word is not cleared, so the handle keeps
// reporting it).  The stage then read its input from global memory, so the
// results are those of a normal step.
static int wait_status(les_handle *h)
{
    if (h->prec != LES_FP32) return LES_OK;
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, h->d_oob, sizeof(v), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if ((v >> 48) == 9)
        return fail(h, LES_ERR_CUDA,
                    "a staging copy of the fused stage did not complete even after the stage stopped "
                    "waiting for it: the state is unreliable");
    if ((v >> 48) == 8)
        return fail(h, LES_ERR_TIMEOUT,
                    "a staging wait of the fused stage gave up (the stage fell back to direct loads)");
    return LES_OK;
}

// ---------------------------------------------------------------------------
// Validation and memory plan
// ---------------------------------------------------------------------------

static void plan_jet(const les_grid_desc *g, int prec, JetHost &J);

static std::string validate(const les_grid_desc *g, const les_params *p)
{
    if (!g || !p) return "null descriptor or parameters";
    if (g->ni < 4 || g->nj < 4 || g->nk < 4) return "each axis needs >= 4 points";
    if (!g->x || !g->y || !g->z) return "null coordinate array";
    if (g->precision != LES_FP64 && g->precision != LES_FP32 && g->precision != LES_FP32_SEPARABLE)
        return "unknown precision";
    if (g->precision != LES_FP64) {
        // the fused FP32 stage addresses the five fields of a register and the
        // static records with 32-bit offsets
        JetHost J;
        plan_jet(g, LES_FP32, J);
        const long long rec = (long long)g->nk * ((g->nj + 1) / 2) * 5 * J.pitch;
        if (5 * J.fs > INT_MAX || rec > INT_MAX)
            return "FP32 grid too large: 5 x padded points (" + std::to_string(5 * J.fs) +
                   ") must stay below 2^31";
    }
    for (int a = 0; a < 3; ++a) {
        bool pf = g->face_bc[2 * a] == LES_BC_PERIODIC, pb = g->face_bc[2 * a + 1] == LES_BC_PERIODIC;
        if (g->periodic[a] != 0 && g->periodic[a] != 1) return "periodic flags must be 0/1";
        if (g->periodic[a] && !(pf && pb)) return "periodic axis needs PERIODIC on both faces";
        if (!g->periodic[a] && (pf || pb)) return "PERIODIC face on a non-periodic axis";
    }
    // the paper's overlapping form of a periodic axis (Sec. "Periodic Boundary
    // Condition": the last plane repeats the first) would give a zero-width
    // cell; this library takes the unique planes only
    {
        const int n[3] = {g->ni, g->nj, g->nk};
        for (int a = 0; a < 3; ++a) {
            if (!g->periodic[a]) continue;
            double dmax = 0.0, ext = 0.0;
            const long long np = (long long)n[0] * n[1] * n[2];
            for (long long l = 0; l < np; ++l) {
                const long long q[3] = {l % n[0], (l / n[0]) % n[1], l / ((long long)n[0] * n[1])};
                if (q[a] != 0) continue;
                long long r[3] = {q[0], q[1], q[2]};
                r[a] = n[a] - 1;
                const long long lr = (r[2] * n[1] + r[1]) * n[0] + r[0];
                const double *X[3] = {g->x, g->y, g->z};
                for (int c = 0; c < 3; ++c) {
                    dmax = std::max(dmax, std::fabs(X[c][lr] - (X[c][l] + g->period_shift[a][c])));
                    ext = std::max(ext, std::fabs(X[c][l]) + std::fabs(g->period_shift[a][c]));
                }
            }
            if (dmax <= 1e-12 * std::max(ext, 1.0))
                return "periodic axis " + std::to_string(a) +
                       " repeats its first plane as its last (overlapping form): pass the unique planes";
        }
    }
    for (int f = 0; f < 6; ++f) {
        int t = g->face_bc[f];
        if (t < LES_BC_PERIODIC || t > LES_BC_CENTERLINE) return "unknown face boundary condition";
        if (t == LES_BC_INFLOW_JET && f != 0) return "INFLOW_JET is allowed on the i- face only";
        if (t == LES_BC_CENTERLINE && f != 2) return "CENTERLINE is allowed on the j- face only";
        if (t == LES_BC_CENTERLINE && !g->periodic[2]) return "CENTERLINE needs a periodic (azimuthal) k axis";
    }
    if (g->face_bc[0] == LES_BC_INFLOW_JET && !(p->mach_j > 0.0)) return "INFLOW_JET needs mach_j > 0";
    if (!(p->gamma > 1.0) || !(p->Pr > 0) || !(p->Pr_sgs > 0) || !(p->Re > 0) || !(p->Cs >= 0) ||
        !(p->k2 >= 0) || !(p->k4 >= 0) || !(p->TR > 0) || !(p->T_inf_dim > 0) || !(p->theta > 0) ||
        !(p->cfl > 0) || !(p->dt >= 0))
        return "invalid flow parameters";
    return "";
}

static void plan_jet(const les_grid_desc *g, int prec, JetHost &J)
{
    const size_t es = prec == LES_FP64 ? 8 : 4;
    J.n[0] = g->ni;
    J.n[1] = g->nj;
    J.n[2] = g->nk;
    const int line = (int)(128 / es);
    J.pitch = (int)align_up((size_t)g->ni, (size_t)line);
    J.npad = (long long)g->nk * g->nj * J.pitch;
    J.fs = (long long)align_up((size_t)J.npad, 64);
    J.N = (long long)g->ni * g->nj * g->nk;
    size_t fb = (size_t)J.fs * es;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = align_up(off + b, 256);
        return o;
    };
    size_t o_met = take((prec == LES_FP64 ? NMET64 : NMET) * fb);
    size_t o_j64 = prec == LES_FP32 ? take((size_t)J.fs * 8) : 0;
    size_t o_q0 = take(NF * fb);
    size_t o_q1 = take(NF * fb);
    size_t o_q2 = take(NF * fb);
    size_t o_prim = take(NPRIM * fb);
    size_t o_grad = take(NGRAD * fb);
    size_t o_hf = take(NHF * fb);
    size_t o_rhs = take(NF * fb);
    size_t o_inr = take((size_t)g->nj * g->nk * 8);
    size_t o_h1 = prec == LES_FP32 ? take((size_t)(g->ni + g->nj + g->nk) * 16) : 0;
    const bool packed = g->precision == LES_FP32; // general FP32 form only
    size_t o_mp = packed ? take((size_t)g->nk * ((g->nj + 1) / 2) * J.pitch * 80) : 0;
    J.bytes = off;
    // store offsets relative to the jet region in the pointers for now
    J.met = (char *)o_met;
    J.jinv64 = prec == LES_FP32 ? (double *)o_j64 : (double *)(o_met + MET_JINV * fb);
    J.q[0] = (char *)o_q0;
    J.q[1] = (char *)o_q1;
    J.q[2] = (char *)o_q2;
    J.prim = (char *)o_prim;
    J.grad = (char *)o_grad;
    J.hflux = (char *)o_hf;
    J.rhs = (char *)o_rhs;
    J.inflow_ut = (double *)o_inr;
    J.h1[0] = prec == LES_FP32 ? (float4 *)o_h1 : nullptr;
    J.h1[1] = prec == LES_FP32 ? (float4 *)(o_h1 + (size_t)g->ni * 16) : nullptr;
    J.h1[2] = prec == LES_FP32 ? (float4 *)(o_h1 + (size_t)(g->ni + g->nj) * 16) : nullptr;
    J.mp = packed ? (float4 *)o_mp : nullptr;
}

// Storage precision of a descriptor's precision code.
static int storage_prec(int precision) { return precision == LES_FP64 ? LES_FP64 : LES_FP32; }

struct GlobalPlan {
    size_t o_jets, o_maps, o_dt, o_level, o_bits, o_part, o_diag, o_pbase, o_stage, o_fj, o_oob, o_tmap, total;
};

static GlobalPlan plan_global(int njets, size_t jetdev_bytes, int nblk_diag, long long maxN)
{
    GlobalPlan P;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = align_up(off + b, 256);
        return o;
    };
    P.o_jets = take(jetdev_bytes * njets);
    P.o_maps = take(sizeof(int) * 4 * (njets + 1) + sizeof(int) * 8 * njets);
    P.o_dt = take(sizeof(double) * njets);
    P.o_level = take(sizeof(long long));
    P.o_bits = take(sizeof(unsigned long long) * njets);
    P.o_part = take(sizeof(double) * 17 * nblk_diag);
    P.o_diag = take(sizeof(double) * 16);
    P.o_pbase = take(sizeof(long long));
    P.o_stage = take(sizeof(double) * 5 * (size_t)maxN);
    P.o_fj = take(sizeof(FusedJet) * 2 * njets);
    P.o_oob = take(sizeof(unsigned long long));
    P.o_tmap = take(sizeof(CUtensorMap) * 6 * njets);
    P.total = off;
    return P;
}

template <typename real> static size_t jetdev_size() { return sizeof(JetDev<real>); }

extern "C" size_t les_workspace_bytes(const les_grid_desc *g)
{
    if (!g || g->ni < 4 || g->nj < 4 || g->nk < 4) return 0;
    JetHost J;
    plan_jet(g, storage_prec(g->precision), J);
    size_t jd = g->precision == LES_FP64 ? jetdev_size<double>() : jetdev_size<float>();
    GlobalPlan P = plan_global(1, jd, DIAG_BLOCKS, J.N);
    return align_up(P.total, 256) + J.bytes;
}

// ---------------------------------------------------------------------------
// Creation
// ---------------------------------------------------------------------------

template <typename real> static void fill_jetdev(const les_handle *h, const JetHost &J, JetDev<real> &D)
{
    std::memset(&D, 0, sizeof(D));
    for (int a = 0; a < 3; ++a) {
        D.n[a] = J.n[a];
        D.per[a] = J.per[a];
    }
    for (int f = 0; f < 6; ++f) D.bc[f] = J.bc[f];
    D.pitch = J.pitch;
    D.fs = J.fs;
    D.npts_pad = J.npad;
    for (int s = 0; s < 3; ++s) D.q[s] = (real *)J.q[s];
    D.met = (const real *)J.met;
    D.jinv64 = J.jinv64;
    D.prim = (real *)J.prim;
    D.grad = (real *)J.grad;
    D.hflux = (real *)J.hflux;
    D.rhs = (real *)J.rhs;
    D.inflow_ut = J.inflow_ut;
    D.oob = h->d_oob;
    const les_params &p = J.prm;
    D.gamma = p.gamma;
    D.Pr = p.Pr;
    D.Pr_sgs = p.Pr_sgs;
    D.Re = p.Re;
    D.mach = p.mach_j;
    D.TR = p.TR;
    D.theta = p.theta;
    D.noise_amp = p.noise_amp;
    D.k2 = p.k2;
    D.k4 = p.k4;
    D.suth_S = p.S1_dim / (p.TR * p.T_inf_dim);
    D.gm1 = p.gamma - 1.0;
    D.suth1 = 1.0 + D.suth_S;
    D.inv_Re = 1.0 / p.Re;
    D.kap_mol = 1.0 / (p.Re * p.Pr * (p.gamma - 1.0));
    D.kap_sgs = 1.0 / (p.Pr_sgs * (p.gamma - 1.0));
    D.bc_g1 = 1.0 / (p.gamma - 1.0);
    D.bc_rg = 1.0 / p.gamma;
    D.bc_cinf = std::sqrt(p.gamma * (1.0 / p.gamma) / p.TR);
    D.seed = (unsigned long long)p.seed;
    (void)h;
}

template <typename real> static int setup_jet(les_handle *h, JetHost &J, const les_grid_desc *g)
{
    const size_t N = (size_t)J.N;
    // temporaries in the (still unused) stage-register / scratch region
    double *tmp = (double *)J.q[1];
    double *dx = tmp, *dy = tmp + N, *dz = tmp + 2 * N;
    CK(cudaMemcpyAsync(dx, g->x, N * 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dy, g->y, N * 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dz, g->z, N * 8, cudaMemcpyHostToDevice, h->st));
    double *met64;
    if (h->prec == LES_FP64)
        met64 = (double *)J.met;
    else
        met64 = (double *)align_up((size_t)(tmp + 3 * N), 256);
    Launch<real>::metrics(dx, dy, dz, J.n[0], J.n[1], J.n[2], J.per, J.shift, met64, J.fs, J.pitch,
                          J.prm.Cs, h->st);
    CK(cudaGetLastError());
    Launch<real>::static_fields(met64, J.fs, J.pitch, J.n, J.per, h->prec == LES_FP64 ? 1 : 0, h->st);
    CK(cudaGetLastError());
    if (h->sep) {
        launch_sep_metrics(dx, dy, dz, J.n, J.per, J.shift, J.h1[0], J.h1[1], J.h1[2], h->st);
        CK(cudaGetLastError());
    }
    if (h->prec == LES_FP32) {
        Launch<real>::convert_metrics(met64, J.fs, (real *)J.met, J.fs, J.npad, h->st);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(J.jinv64, met64 + MET_JINV * J.fs, (size_t)J.fs * 8,
                           cudaMemcpyDeviceToDevice, h->st));
        if (J.mp) {
            launch_pack_pairs((const float *)J.met, J.fs, J.pitch, J.n[1], J.n[2], J.mp, h->st);
            CK(cudaGetLastError());
        }
    }
    // inflow profile u~(r) = [1 + tanh((0.5 - r)/(2 theta))]/2 of the
    // inflow-face points, r = (y^2 + z^2)^1/2 (static: formed once here)
    std::vector<double> ut((size_t)J.n[1] * J.n[2]);
    for (int k = 0; k < J.n[2]; ++k)
        for (int j = 0; j < J.n[1]; ++j) {
            size_t p = ((size_t)k * J.n[1] + j) * J.n[0];
            const double r = std::sqrt(g->y[p] * g->y[p] + g->z[p] * g->z[p]);
            ut[(size_t)k * J.n[1] + j] = 0.5 * (1.0 + std::tanh((0.5 - r) / (2.0 * J.prm.theta)));
        }
    CK(cudaMemcpyAsync(J.inflow_ut, ut.data(), ut.size() * 8, cudaMemcpyHostToDevice, h->st));
    // positive cell volumes
    std::vector<double> jv((size_t)J.fs);
    CK(cudaMemcpyAsync(jv.data(), J.jinv64, (size_t)J.fs * 8, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    const bool axis = J.bc[2] == LES_BC_CENTERLINE;
    for (int k = 0; k < J.n[2]; ++k)
        for (int j = 0; j < J.n[1]; ++j)
            for (int i = 0; i < J.n[0]; ++i) {
                double v = jv[((size_t)k * J.n[1] + j) * J.pitch + i];
                if (axis && j == 0 && v == 0.0) continue; // the degenerate axis of a polar mesh
                if (!(v > 0.0) || !std::isfinite(v))
                    return fail(h, LES_ERR_ARG, "non-positive or non-finite cell volume J^-1 at (" +
                                                    std::to_string(i) + "," + std::to_string(j) +
                                                    "," + std::to_string(k) + ")");
            }
    // product-grid detection (probe)
    J.product = true;
    for (size_t p = 0; p < N && J.product; ++p) {
        size_t i = p % J.n[0], j = (p / J.n[0]) % J.n[1], k = p / ((size_t)J.n[0] * J.n[1]);
        if (g->x[p] != g->x[i] || g->y[p] != g->y[j * J.n[0]] ||
            g->z[p] != g->z[k * (size_t)J.n[0] * J.n[1]])
            J.product = false;
    }
    if (h->sep && !J.product)
        return fail(h, LES_ERR_ARG, "LES_FP32_SEPARABLE needs a Cartesian-product grid x(i), y(j), z(k)");
    if (J.product) {
        for (int i = 0; i < J.n[0]; ++i) J.ax[0].push_back(g->x[i]);
        for (int j = 0; j < J.n[1]; ++j) J.ax[1].push_back(g->y[(size_t)j * J.n[0]]);
        for (int k = 0; k < J.n[2]; ++k) J.ax[2].push_back(g->z[(size_t)k * J.n[0] * J.n[1]]);
    }
    return LES_OK;
}

// Interior output range length of one axis.
static int out_len(const JetHost &J, int a) { return J.per[a] ? J.n[a] : J.n[a] - 2; }

// Work-list tables of the fused stage for tile height ty and k-chunk kc
// (kc = 0: balanced form, items are tile-planes split evenly over the grid;
// kc = -1: the same after waves of whole columns, in lockstep).
static int set_fused_tiling(les_handle *h, int ty, int kc)
{
    int acc = 0, tiles = 0;
    std::vector<FusedJet> one(h->njets);
    for (int j = 0; j < h->njets; ++j) {
        FusedJet &F = h->fj[j];
        const JetHost &J = h->J[j];
        F.nbx = (out_len(J, 0) + 29) / 30;
        F.nby = (out_len(J, 1) + ty - 3) / (ty - 2);
        if (kc <= 0) {
            F.kc = 0;
            F.nkc = out_len(J, 2); // planes per column: the items are tile-planes
        } else {
            F.kc = std::max(1, std::min(kc, out_len(J, 2)));
            F.nkc = (out_len(J, 2) + F.kc - 1) / F.kc;
        }
        F.item0 = acc;
        F.tile0 = tiles;
        acc += F.nbx * F.nby * F.nkc;
        tiles += F.nbx * F.nby;
        one[j] = F;
        one[j].item0 = 0;
        one[j].tile0 = 0;
    }
    h->fused_ty = ty;
    h->fused_balanced = kc == 0 ? 1 : (kc < 0 ? 2 : 0);
    h->fused_items = acc;
    h->fused_tiles = tiles;
    CK(cudaMemcpyAsync(h->d_fj, h->fj.data(), sizeof(FusedJet) * h->njets, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->d_fj1, one.data(), sizeof(FusedJet) * h->njets, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->fj1 = one;
    return LES_OK;
}

static int items_of(const FusedJet &F) { return F.nbx * F.nby * F.nkc; }
static std::string kc_label(int kc)
{
    return kc == 0 ? std::string("balanced") : (kc < 0 ? std::string("lockstep") : std::to_string(kc));
}
static int autotune_fused(les_handle *h);

// One fused stage (or residual) over all jets (jet < 0) or one jet.
static void fused_launch(les_handle *h, int jet, int src, int dst, int stage, int rhs_only, cudaStream_t st)
{
    const JetDev<float> *jets = (const JetDev<float> *)h->d_jets;
    const FusedJet *fj = jet < 0 ? h->d_fj : h->d_fj1 + jet;
    const int nj = jet < 0 ? h->njets : 1;
    const int items = jet < 0 ? h->fused_items : items_of(h->fj[jet]);
    const int tiles = jet < 0 ? h->fused_tiles : h->fj[jet].nbx * h->fj[jet].nby;
    const int grid = std::max(1, std::min(items, h->nsm * h->fused_cps[h->fused_ty == 16 ? 1 : 0]));
    if (jet >= 0) jets += jet;
    const int bal = h->fused_balanced;
    // a single jet's table entries travel as kernel parameters
    const JetDev<float> *j1 = nj == 1 ? &h->jd32[jet < 0 ? 0 : jet] : nullptr;
    const FusedJet *f1 = nj == 1 ? (jet < 0 ? &h->fj[0] : &h->fj1[jet]) : nullptr;
    if (h->fused_ty == 16)
        launch_fused<16>(jets, fj, nj, items, tiles, grid, src, dst, stage, h->d_dt, rhs_only, h->sep, bal,
                         h->stage_wait_limit, j1, f1, st);
    else
        launch_fused<8>(jets, fj, nj, items, tiles, grid, src, dst, stage, h->d_dt, rhs_only, h->sep, bal,
                         h->stage_wait_limit, j1, f1, st);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links no driver library); null if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    return fn;
}

// TMA maps of one FP32 jet's three state registers for the fused stage's
// staging box (5 fields x 1 plane x (TY + 4) rows x 40 columns) at TY = 8 and
// 16: tensor [field][k][j][i] with the padded row and field strides, columns
// beyond ni read as zero.  Returns false if the encoder refuses.
static bool make_state_maps(const JetHost &J, CUtensorMap out[6])
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)J.n[0], (cuuint64_t)J.n[1], (cuuint64_t)J.n[2], 5};
    const cuuint64_t strides[3] = {(cuuint64_t)J.pitch * 4, (cuuint64_t)J.pitch * J.n[1] * 4, (cuuint64_t)J.fs * 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int t = 0; t < 2; ++t) {
        const cuuint32_t box[4] = {(cuuint32_t)TMA_BOX_X, (cuuint32_t)tma_box_rows(t == 0 ? 8 : 16), 1, 5};
        for (int r = 0; r < 3; ++r)
            if (enc(&out[3 * t + r], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, J.q[r], dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
    }
    return true;
}

template <typename real>
static int create_impl(const les_grid_desc *g, const les_params *p, int njets, void *stream,
                       les_handle **out)
{
    les_handle *h = new les_handle();
    h->prec = storage_prec(g[0].precision);
    h->sep = g[0].precision == LES_FP32_SEPARABLE;
    h->njets = njets;
    h->st = (cudaStream_t)stream;
    auto bail = [&](int code) {
        g_create_err = h->err;
        les_destroy(h);
        *out = nullptr;
        return code;
    };
    CK(cudaGetDevice(&h->dev));
    CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
    CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    h->J.resize(njets);
    long long maxN = 0;
    size_t jets_bytes = 0;
    for (int j = 0; j < njets; ++j) {
        JetHost &J = h->J[j];
        plan_jet(&g[j], h->prec, J);
        J.prm = p[j];
        for (int a = 0; a < 3; ++a) J.per[a] = g[j].periodic[a];
        for (int f = 0; f < 6; ++f) J.bc[f] = g[j].face_bc[f];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) J.shift[3 * a + c] = g[j].period_shift[a][c];
        J.nblk_pt = (int)((J.npad + BLOCK - 1) / BLOCK);
        for (int a = 0; a < 3; ++a) {
            if (J.per[a]) {
                J.nblk_bc[a] = 0;
                continue;
            }
            long long nface = (long long)J.n[(a + 1) % 3] * J.n[(a + 2) % 3];
            J.nblk_bc[a] = (int)((2 * nface + BLOCK - 1) / BLOCK);
        }
        J.off = jets_bytes;
        jets_bytes += align_up(J.bytes, 256);
        maxN = std::max(maxN, J.N);
        if (J.bc[2] == LES_BC_CENTERLINE) h->centerline = true;
        h->max_ni = std::max(h->max_ni, J.n[0]);
    }
    h->nblk_diag = DIAG_BLOCKS;
    GlobalPlan GP = plan_global(njets, sizeof(JetDev<real>), h->nblk_diag, maxN);
    size_t gbytes = align_up(GP.total, 256);
    h->bytes = gbytes + jets_bytes;
    if (njets == 1 && g[0].workspace) {
        if (((uintptr_t)g[0].workspace & 255) != 0 || g[0].workspace_bytes < h->bytes) {
            fail(h, LES_ERR_OOM, "workspace too small or not 256-byte aligned");
            return bail(LES_ERR_OOM);
        }
        h->base = (char *)g[0].workspace;
        h->owns = false;
    } else {
        if (cudaMalloc((void **)&h->base, h->bytes) != cudaSuccess) {
            cudaGetLastError();
            h->base = nullptr;
            fail(h, LES_ERR_OOM, "cudaMalloc of " + std::to_string(h->bytes) + " bytes failed");
            return bail(LES_ERR_OOM);
        }
        h->owns = true;
    }
    char *B = h->base;
    h->d_jets = B + GP.o_jets;
    h->d_maps = (int *)(B + GP.o_maps);
    h->d_dt = (double *)(B + GP.o_dt);
    h->d_level = (long long *)(B + GP.o_level);
    h->d_dtbits = (unsigned long long *)(B + GP.o_bits);
    h->d_partials = (double *)(B + GP.o_part);
    h->d_diag = (double *)(B + GP.o_diag);
    h->d_probe_base = (long long *)(B + GP.o_pbase);
    h->d_stage = (double *)(B + GP.o_stage);
    h->d_fj = (FusedJet *)(B + GP.o_fj);
    h->d_oob = (unsigned long long *)(B + GP.o_oob);
    h->d_tmap = (CUtensorMap *)(B + GP.o_tmap);
    h->d_fj1 = h->d_fj + njets;
    for (int j = 0; j < njets; ++j) {
        JetHost &J = h->J[j];
        char *jb = B + gbytes + J.off;
        J.met = jb + (size_t)J.met;
        J.jinv64 = (double *)(jb + (size_t)J.jinv64);
        for (int s = 0; s < 3; ++s) J.q[s] = jb + (size_t)J.q[s];
        J.prim = jb + (size_t)J.prim;
        J.grad = jb + (size_t)J.grad;
        J.hflux = jb + (size_t)J.hflux;
        J.rhs = jb + (size_t)J.rhs;
        J.inflow_ut = (double *)(jb + (size_t)J.inflow_ut);
        for (int a = 0; a < 3; ++a)
            if (J.h1[a]) J.h1[a] = (float4 *)(jb + (size_t)J.h1[a]);
        if (J.mp) J.mp = (float4 *)(jb + (size_t)J.mp);
    }
    for (int j = 0; j < njets; ++j) {
        int rc = setup_jet<real>(h, h->J[j], &g[j]);
        if (rc != LES_OK) return bail(rc);
    }
    // device jet table
    std::vector<JetDev<real>> D(njets);
    for (int j = 0; j < njets; ++j) fill_jetdev<real>(h, h->J[j], D[j]);
    CK(cudaMemcpyAsync(h->d_jets, D.data(), sizeof(JetDev<real>) * njets, cudaMemcpyHostToDevice, h->st));
    if constexpr (sizeof(real) == sizeof(float)) h->jd32 = D;
    if (h->prec == LES_FP32) {
        if (fused_prepare<16>() != 0 || fused_prepare<8>() != 0)
            return bail(fail(h, LES_ERR_CUDA, "fused kernel shared-memory attribute"));
        h->fused_cps[0] = fused_ctas_per_sm(8, h->sep ? 1 : 0);
        h->fused_cps[1] = fused_ctas_per_sm(16, h->sep ? 1 : 0);
        h->fj.resize(njets);
        for (int j = 0; j < njets; ++j) {
            FusedParams &F = h->fj[j].fp;
            const les_params &pp = h->J[j].prm;
            F.gam = (float)pp.gamma;
            F.gm1 = (float)(pp.gamma - 1.0);
            F.hgam = (float)(pp.gamma / (pp.gamma - 1.0));
            F.k2 = (float)pp.k2;
            F.k4 = (float)pp.k4;
            F.inv_Re = (float)(1.0 / pp.Re);
            F.kap_mol = (float)(1.0 / (pp.Re * pp.Pr * (pp.gamma - 1.0)));
            F.kap_sgs = (float)(1.0 / (pp.Pr_sgs * (pp.gamma - 1.0)));
            const double S = pp.S1_dim / (pp.TR * pp.T_inf_dim);
            F.suth1 = (float)(1.0 + S);
            F.suthS = (float)S;
            F.cs2 = (float)(pp.Cs * pp.Cs);
            F.pinf = (float)(1.0 / pp.gamma);
            for (int a = 0; a < 3; ++a) h->fj[j].h1[a] = h->J[j].h1[a];
            h->fj[j].mp = h->J[j].mp;
            h->fj[j].njp = (h->J[j].n[1] + 1) / 2;
            h->fj[j].tmap = nullptr;
        }
        // TMA maps for jets whose i and j axes are not periodic (a periodic
        // tile halo wraps, which a box cannot)
        {
            std::vector<CUtensorMap> maps(6 * (size_t)njets);
            std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
            for (int j = 0; j < njets; ++j)
                if (!h->J[j].per[0] && !h->J[j].per[1] && make_state_maps(h->J[j], &maps[6 * (size_t)j]))
                    h->fj[j].tmap = h->d_tmap + 6 * (size_t)j;
            CK(cudaMemcpyAsync(h->d_tmap, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                               h->st));
        }
        int rc = set_fused_tiling(h, 8, 32);
        if (rc) return bail(rc);
    }
    // block maps: [pt | bc0 | bc1 | bc2] each njets+1, then per-jet pairs
    std::vector<int> maps(4 * (njets + 1) + 8 * njets);
    for (int fam = 0; fam < 4; ++fam) {
        int acc = 0;
        for (int j = 0; j < njets; ++j) {
            maps[fam * (njets + 1) + j] = acc;
            acc += fam == 0 ? h->J[j].nblk_pt : h->J[j].nblk_bc[fam - 1];
        }
        maps[fam * (njets + 1) + njets] = acc;
        BlockMap bm{h->d_maps + fam * (njets + 1), njets, acc};
        if (fam == 0) h->pt = bm; else h->bcm[fam - 1] = bm;
    }
    int *pj = maps.data() + 4 * (njets + 1);
    h->pt1.resize(njets);
    for (int a = 0; a < 3; ++a) h->bc1[a].resize(njets);
    for (int j = 0; j < njets; ++j) {
        for (int fam = 0; fam < 4; ++fam) {
            int nb = fam == 0 ? h->J[j].nblk_pt : h->J[j].nblk_bc[fam - 1];
            pj[8 * j + 2 * fam] = 0;
            pj[8 * j + 2 * fam + 1] = nb;
            BlockMap bm{h->d_maps + 4 * (njets + 1) + 8 * j + 2 * fam, 1, nb};
            if (fam == 0) h->pt1[j] = bm; else h->bc1[fam - 1][j] = bm;
        }
    }
    CK(cudaMemcpyAsync(h->d_maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->d_level, 0, sizeof(long long), h->st));
    CK(cudaMemsetAsync(h->d_oob, 0, sizeof(unsigned long long), h->st));
    CK(cudaMemsetAsync(h->d_dt, 0, sizeof(double) * njets, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->dt.assign(njets, 0.0);
    h->has_state.assign(njets, 0);
    for (int j = 0; j < njets; ++j)
        if (p[j].dt > 0) h->dt[j] = p[j].dt;
    CK(cudaMemcpyAsync(h->d_dt, h->dt.data(), sizeof(double) * njets, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    *out = h;
    return LES_OK;
}

static int create_any(const les_grid_desc *g, const les_params *p, int njets, void *stream,
                      les_handle **out)
{
    g_create_err.clear();
    if (!out) {
        g_create_err = "null output pointer";
        return LES_ERR_ARG;
    }
    *out = nullptr;
    if (!g || !p || njets < 1) {
        g_create_err = "null descriptor or parameters, or njets < 1";
        return LES_ERR_ARG;
    }
    for (int j = 0; j < njets; ++j) {
        std::string msg = validate(&g[j], &p[j]);
        if (!msg.empty()) {
            g_create_err = "jet " + std::to_string(j) + ": " + msg;
            return LES_ERR_ARG;
        }
        if (g[j].precision != g[0].precision) {
            g_create_err = "all jets of a batch need the same precision";
            return LES_ERR_ARG;
        }
    }
    if (g[0].precision == LES_FP64) return create_impl<double>(g, p, njets, stream, out);
    return create_impl<float>(g, p, njets, stream, out);
}

extern "C" int les_create_grid(const les_grid_desc *g, const les_params *p, void *stream,
                               les_handle **out)
{
    return create_any(g, p, 1, stream, out);
}

extern "C" int les_create_batch(const les_grid_desc *g, const les_params *p, int njets, void *stream,
                                les_handle **out)
{
    if (!g) return LES_ERR_ARG;
    std::vector<les_grid_desc> gg(g, g + std::max(njets, 0));
    for (auto &d : gg) {
        d.workspace = nullptr;
        d.workspace_bytes = 0;
    }
    return create_any(gg.data(), p, njets, stream, out);
}

// ---------------------------------------------------------------------------
// Stage sequence
// ---------------------------------------------------------------------------

static int grid_cap(les_handle *h, int total) { return std::max(1, std::min(total, h->nsm * 8)); }

template <typename real>
static int rhs_pass(les_handle *h, const BlockMap &pt, const JetDev<real> *jets, int src,
                    int rhs_only, int dst, int stage)
{
    // the four-kernel stage needs the FP64 interface tables
    if (h->prec != LES_FP64) return fail(h, LES_ERR_STATE, "four-kernel stage on an FP32 handle");
    int gp = grid_cap(h, pt.total);
    Launch<real>::point(jets, pt, src, gp, h->st);
    Launch<real>::grads(jets, pt, gp, h->st);
    Launch<real>::iface(jets, pt, gp, h->st);
    Launch<real>::update(jets, pt, dst, stage, h->d_dt, rhs_only, gp, h->st);
    CK(cudaGetLastError());
    return LES_OK;
}

template <typename real>
static int bc_pass(les_handle *h, const BlockMap bcm[3], const JetDev<real> *jets, int dst,
                   cudaStream_t st)
{
    static const int order[3] = {1, 2, 0};
    for (int oi = 0; oi < 3; ++oi) {
        int a = order[oi];
        if (a == 1 && h->centerline) {
            launch_centerline<real>(jets, bcm[1].njets, h->max_ni, dst, st);
            h->launches_per_step++;
        }
        if (bcm[a].total == 0) continue;
        Launch<real>::bc(jets, bcm[a], a, dst, h->d_level, grid_cap(h, bcm[a].total), st);
        h->launches_per_step++;
    }
    CK(cudaGetLastError());
    return LES_OK;
}

// Optional per-launch event timing (les_profile_step); inactive during capture.
struct Tracer {
    bool on = false;
    cudaStream_t st = nullptr; // may be the legacy default stream (NULL)
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    void begin(int kind)
    {
        if (!on) return;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        ev.push_back({kind, {a, b}});
    }
    void end()
    {
        if (!on) return;
        cudaEventRecord(ev.back().second.second, st);
    }
};

template <typename real> static int record_step(les_handle *h, cudaStream_t st, Tracer *tr = nullptr)
{
    Tracer none;
    Tracer &T = tr ? *tr : none;
    const JetDev<real> *jets = (const JetDev<real> *)h->d_jets;
    static const int src_of[5] = {0, 1, 2, 1, 2};
    static const int dst_of[5] = {1, 2, 1, 2, 0};
    static const int order[3] = {1, 2, 0};
    h->launches_per_step = 0;
    T.begin(LES_KERNEL_OTHER);
    launch_step_advance(h->d_level, st);
    T.end();
    h->launches_per_step++;
    int gp = grid_cap(h, h->pt.total);
    for (int s = 0; s < 5; ++s) {
        if (h->prec == LES_FP32) {
            // fused single-pass stage: counted as the interface kernel kind
            T.begin(LES_KERNEL_IFACE);
            fused_launch(h, -1, src_of[s], dst_of[s], s, 0, st);
            T.end();
            h->launches_per_step += 1;
            for (int oi = 0; oi < 3; ++oi) {
                int a = order[oi];
                if (a == 1 && h->centerline) {
                    T.begin(LES_KERNEL_BC);
                    launch_centerline<real>(jets, h->njets, h->max_ni, dst_of[s], st);
                    T.end();
                    h->launches_per_step++;
                }
                if (h->bcm[a].total == 0) continue;
                T.begin(LES_KERNEL_BC);
                Launch<real>::bc(jets, h->bcm[a], a, dst_of[s], h->d_level, grid_cap(h, h->bcm[a].total), st);
                T.end();
                h->launches_per_step++;
            }
            continue;
        }
        T.begin(LES_KERNEL_POINT);
        Launch<real>::point(jets, h->pt, src_of[s], gp, st);
        T.end();
        T.begin(LES_KERNEL_GRADS);
        Launch<real>::grads(jets, h->pt, gp, st);
        T.end();
        T.begin(LES_KERNEL_IFACE);
        Launch<real>::iface(jets, h->pt, gp, st);
        T.end();
        T.begin(LES_KERNEL_UPDATE);
        Launch<real>::update(jets, h->pt, dst_of[s], s, h->d_dt, 0, gp, st);
        T.end();
        h->launches_per_step += 4;
        for (int oi = 0; oi < 3; ++oi) {
            int a = order[oi];
            if (a == 1 && h->centerline) {
                T.begin(LES_KERNEL_BC);
                launch_centerline<real>(jets, h->njets, h->max_ni, dst_of[s], st);
                T.end();
                h->launches_per_step++;
            }
            if (h->bcm[a].total == 0) continue;
            T.begin(LES_KERNEL_BC);
            Launch<real>::bc(jets, h->bcm[a], a, dst_of[s], h->d_level, grid_cap(h, h->bcm[a].total), st);
            T.end();
            h->launches_per_step++;
        }
    }
    if (h->probe_npts > 0) {
        T.begin(LES_KERNEL_OTHER);
        Launch<real>::probe(jets, h->d_cell, h->d_wts, h->probe_npts, h->probe_every, h->d_level,
                            h->d_probe_base, (real *)h->probe_out, h->probe_cap, st);
        T.end();
        h->launches_per_step++;
    }
    CK(cudaGetLastError());
    return LES_OK;
}

template <typename real> static int profile_impl(les_handle *h, int nsteps, double *ms, int64_t *cnt)
{
    for (int k = 0; k < LES_KERNEL_KINDS; ++k) {
        ms[k] = 0.0;
        if (cnt) cnt[k] = 0;
    }
    for (int s = 0; s < nsteps; ++s) {
        Tracer tr;
        tr.on = true;
        tr.st = h->st;
        int rc = record_step<real>(h, h->st, &tr);
        CK(cudaStreamSynchronize(h->st));
        for (auto &e : tr.ev) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e.second.first, e.second.second);
            ms[e.first] += t;
            if (cnt) cnt[e.first]++;
            cudaEventDestroy(e.second.first);
            cudaEventDestroy(e.second.second);
        }
        if (rc) return rc;
        h->step += 1;
    }
    return LES_OK;
}

extern "C" int les_profile_step(les_handle *h, int nsteps, double *ms_out, int64_t *counts)
{
    if (!h || nsteps < 0 || !ms_out) return LES_ERR_ARG;
    for (int j = 0; j < h->njets; ++j)
        if (!h->has_state[j]) return fail(h, LES_ERR_STATE, "les_profile_step before les_set_state");
    if (h->prec == LES_FP32 && !h->tuned) {
        int rc = autotune_fused(h);
        if (rc) return rc;
        h->tuned = true;
    }
    return h->prec == LES_FP64 ? profile_impl<double>(h, nsteps, ms_out, counts)
                               : profile_impl<float>(h, nsteps, ms_out, counts);
}

template <typename real> static int capture_step(les_handle *h)
{
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int rc = record_step<real>(h, h->cap);
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (rc != LES_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(h, LES_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(h, LES_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return LES_OK;
}

extern "C" int les_step(les_handle *h, int nsteps)
{
    if (!h || nsteps < 0) return LES_ERR_ARG;
    for (int j = 0; j < h->njets; ++j)
        if (!h->has_state[j]) return fail(h, LES_ERR_STATE, "les_step before les_set_state");
    if (h->prec == LES_FP32 && !h->tuned) {
        int rc = autotune_fused(h);
        if (rc) return rc;
        h->tuned = true;
    }
    if (!h->gexec) {
        int rc = h->prec == LES_FP64 ? capture_step<double>(h) : capture_step<float>(h);
        if (rc) return rc;
    }
    for (int s = 0; s < nsteps; ++s) CK(cudaGraphLaunch(h->gexec, h->st));
    h->step += nsteps;
    h->last_launches = (int64_t)nsteps * h->launches_per_step;
    return LES_OK;
}

// ---------------------------------------------------------------------------
// State transfer, time, diagnostics
// ---------------------------------------------------------------------------

static bool bad_jet(les_handle *h, int jet) { return !h || jet < 0 || jet >= h->njets; }

template <typename real> static int set_state_impl(les_handle *h, int jet, const double *q, int kind)
{
    JetHost &J = h->J[jet];
    const JetDev<real> *jets = (const JetDev<real> *)h->d_jets;
    CK(cudaMemcpyAsync(h->d_stage, q, (size_t)J.N * 5 * 8, cudaMemcpyHostToDevice, h->st));
    Launch<real>::set_state(jets, jet, h->d_stage, kind, J.npad, h->st);
    CK(cudaGetLastError());
    // boundary conditions of the current level on this jet (faces y, z, x)
    const JetDev<real> *one = jets + jet;
    BlockMap b1[3] = {h->bc1[0][jet], h->bc1[1][jet], h->bc1[2][jet]};
    int64_t saved = h->launches_per_step;
    int rc = bc_pass<real>(h, b1, one, 0, h->st);
    h->launches_per_step = saved;
    if (rc) return rc;
    if (h->dt[jet] == 0.0) {
        BlockMap p1 = h->pt1[jet];
        Launch<real>::point(one, p1, 0, grid_cap(h, p1.total), h->st);
        CK(cudaMemsetAsync(h->d_dtbits + jet, 0, 8, h->st));
        Launch<real>::dt_max(one, p1, h->d_dtbits + jet, grid_cap(h, p1.total), h->st);
        CK(cudaGetLastError());
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, h->d_dtbits + jet, 8, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        double mx;
        std::memcpy(&mx, &bits, 8);
        if (!(mx > 0.0) || !std::isfinite(mx)) return fail(h, LES_ERR_NONFINITE, "invalid spectral radius in state");
        h->dt[jet] = J.prm.cfl / mx;
        CK(cudaMemcpyAsync(h->d_dt + jet, &h->dt[jet], 8, cudaMemcpyHostToDevice, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    h->has_state[jet] = 1;
    return LES_OK;
}

extern "C" int les_set_state_jet(les_handle *h, int jet, const double *q, int kind)
{
    if (bad_jet(h, jet) || !q || kind < 0 || kind > 2) return LES_ERR_ARG;
    return h->prec == LES_FP64 ? set_state_impl<double>(h, jet, q, kind)
                               : set_state_impl<float>(h, jet, q, kind);
}

extern "C" int les_set_state(les_handle *h, const double *q, int kind)
{
    return les_set_state_jet(h, 0, q, kind);
}

template <typename real> static int get_state_impl(les_handle *h, int jet, double *q, int kind)
{
    JetHost &J = h->J[jet];
    const JetDev<real> *jets = (const JetDev<real> *)h->d_jets;
    Launch<real>::get_state(jets, jet, h->d_stage, kind, J.npad, h->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(q, h->d_stage, (size_t)J.N * 5 * 8, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return wait_status(h);
}

extern "C" int les_get_state_jet(les_handle *h, int jet, double *q, int kind)
{
    if (bad_jet(h, jet) || !q || kind < 0 || kind > 2) return LES_ERR_ARG;
    return h->prec == LES_FP64 ? get_state_impl<double>(h, jet, q, kind)
                               : get_state_impl<float>(h, jet, q, kind);
}

extern "C" int les_get_state(les_handle *h, double *q, int kind) { return les_get_state_jet(h, 0, q, kind); }

extern "C" int les_set_time(les_handle *h, int64_t step, double dt)
{
    if (!h || step < 0 || !(dt > 0)) return LES_ERR_ARG;
    h->step = step;
    long long lv = step;
    for (int j = 0; j < h->njets; ++j) h->dt[j] = dt;
    CK(cudaMemcpyAsync(h->d_level, &lv, 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->d_dt, h->dt.data(), 8 * h->njets, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LES_OK;
}

extern "C" int les_get_time(les_handle *h, int64_t *step, double *dt)
{
    if (!h) return LES_ERR_ARG;
    if (step) *step = h->step;
    if (dt) *dt = h->dt[0];
    return LES_OK;
}

template <typename real> static int residual_of_jet(les_handle *h, int jet)
{
    if (h->prec == LES_FP32) {
        // the same fused kernel as the steps; it writes interior points only
        JetHost &J = h->J[jet];
        CK(cudaMemsetAsync(J.rhs, 0, (size_t)J.fs * NF * sizeof(float), h->st));
        fused_launch(h, jet, 0, 0, 0, 1, h->st);
        CK(cudaGetLastError());
        return LES_OK;
    }
    const JetDev<real> *one = (const JetDev<real> *)h->d_jets + jet;
    return rhs_pass<real>(h, h->pt1[jet], one, 0, 1, 0, 0);
}

// Autotuner of the fused stage: time (tile height, k-chunk) candidates with
// real stage launches on the current state and keep the fastest; the choice
// is cached per device and set of grid shapes for the process (under a lock:
// handles may be stepped from several host threads; the timing itself runs
// outside it, so two threads may tune the same key, and the first result
// stays).
static std::map<std::string, std::pair<int, int>> g_tune_cache;
static std::mutex g_tune_mu;

namespace {
struct EventPair { // destroyed on every return path
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};
} // namespace

static int autotune_fused(les_handle *h)
{
    std::string key = "dev" + std::to_string(h->dev) + ":";
    for (auto &J : h->J)
        key += std::to_string(J.n[0]) + "x" + std::to_string(J.n[1]) + "x" + std::to_string(J.n[2]) + "p" +
               std::to_string(J.per[0] * 4 + J.per[1] * 2 + J.per[2]) + (h->sep ? "s;" : ";");
    std::pair<int, int> pick{8, 48};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            pick = it->second;
            cached = true;
        }
    }
    if (!cached) {
        const int tys[2] = {16, 8};
        // 0: balanced tile-plane ranges; -1: whole-column waves, then balanced ranges
        const int kcs[8] = {8, 16, 24, 48, 96, 100000, 0, -1};
        float best = 1e30f;
        EventPair ev;
        CK(cudaEventCreate(&ev.e0));
        CK(cudaEventCreate(&ev.e1));
        for (int ty : tys)
            for (int kc : kcs) {
                int rc = set_fused_tiling(h, ty, kc);
                if (rc) return rc;
                // real stage launches from Q(0) into the first stage register,
                // which holds no state between steps
                fused_launch(h, -1, 0, 1, 0, 0, h->st); // warm-up
                CK(cudaEventRecord(ev.e0, h->st));
                for (int rep = 0; rep < 3; ++rep) fused_launch(h, -1, 0, 1, 0, 0, h->st);
                CK(cudaEventRecord(ev.e1, h->st));
                CK(cudaEventSynchronize(ev.e1));
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
                if (ms < best) {
                    best = ms;
                    pick = {ty, kc};
                }
            }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        pick = g_tune_cache.emplace(key, pick).first->second;
    }
    h->tune_note = "ty=" + std::to_string(pick.first) + " kc=" + kc_label(pick.second) +
                   " (tuned over ty {16,8} x kc {8,16,24,48,96,all,balanced,lockstep})";
    return set_fused_tiling(h, pick.first, pick.second);
}

template <typename real> static int diag_impl(les_handle *h, int jet, les_diag *d)
{
    int rc = residual_of_jet<real>(h, jet);
    if (rc) return rc;
    const JetDev<real> *jets = (const JetDev<real> *)h->d_jets;
    Launch<real>::diag_partials(jets, jet, h->d_partials, h->nblk_diag, h->st);
    launch_diag_final(h->d_partials, h->nblk_diag, h->d_diag, h->st);
    CK(cudaGetLastError());
    double out[12];
    CK(cudaMemcpyAsync(out, h->d_diag, sizeof(out), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    d->dt = h->dt[jet];
    d->step = h->step;
    d->max_abs_rhs_rho = out[0];
    for (int f = 0; f < 5; ++f) {
        d->l2_rhs[f] = out[1 + f];
        d->sum_qhat[f] = out[6 + f];
    }
    d->nonfinite = (int64_t)out[11];
    if (int rc = wait_status(h)) return rc;
    if (d->nonfinite > 0 || !std::isfinite(out[0])) return fail(h, LES_ERR_NONFINITE, "non-finite values in state or residual");
    return LES_OK;
}

extern "C" int les_get_diagnostics_jet(les_handle *h, int jet, les_diag *d)
{
    if (bad_jet(h, jet) || !d) return LES_ERR_ARG;
    if (!h->has_state[jet]) return fail(h, LES_ERR_STATE, "no state");
    return h->prec == LES_FP64 ? diag_impl<double>(h, jet, d) : diag_impl<float>(h, jet, d);
}

extern "C" int les_get_diagnostics(les_handle *h, les_diag *d) { return les_get_diagnostics_jet(h, 0, d); }

template <typename real> static int export_impl(les_handle *h, int jet, int field, double *out, size_t n)
{
    JetHost &J = h->J[jet];
    const JetDev<real> *jets = (const JetDev<real> *)h->d_jets;
    Launch<real>::debug_field(jets, jet, field, h->d_stage, J.npad, h->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, h->d_stage, n * 8, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LES_OK;
}

extern "C" int les_debug_rhs(les_handle *h, int jet, double *rhs)
{
    if (bad_jet(h, jet) || !rhs) return LES_ERR_ARG;
    if (!h->has_state[jet]) return fail(h, LES_ERR_STATE, "no state");
    int rc = h->prec == LES_FP64 ? residual_of_jet<double>(h, jet) : residual_of_jet<float>(h, jet);
    if (rc) return rc;
    size_t N = (size_t)h->J[jet].N;
    return h->prec == LES_FP64 ? export_impl<double>(h, jet, DBG_RHS, rhs, 5 * N)
                               : export_impl<float>(h, jet, DBG_RHS, rhs, 5 * N);
}

extern "C" int les_debug_field(les_handle *h, int jet, int field, double *out)
{
    if (bad_jet(h, jet) || !out || field < 0 || field > LES_FIELD_METRICS) return LES_ERR_ARG;
    size_t N = (size_t)h->J[jet].N;
    if (field == LES_FIELD_METRICS) {
        for (int t = 0; t < 10; ++t) {
            int rc = h->prec == LES_FP64 ? export_impl<double>(h, jet, DBG_MET0 + t, out + t * N, N)
                                         : export_impl<float>(h, jet, DBG_MET0 + t, out + t * N, N);
            if (rc) return rc;
        }
        return LES_OK;
    }
    if (!h->has_state[jet]) return fail(h, LES_ERR_STATE, "no state");
    int rc;
    if (h->prec == LES_FP64) {
        const JetDev<double> *one = (const JetDev<double> *)h->d_jets + jet;
        int gp = grid_cap(h, h->pt1[jet].total);
        Launch<double>::point(one, h->pt1[jet], 0, gp, h->st);
        Launch<double>::grads(one, h->pt1[jet], gp, h->st);
        rc = export_impl<double>(h, jet, field, out, N);
    } else {
        const JetDev<float> *one = (const JetDev<float> *)h->d_jets + jet;
        int gp = grid_cap(h, h->pt1[jet].total);
        Launch<float>::point(one, h->pt1[jet], 0, gp, h->st);
        Launch<float>::grads(one, h->pt1[jet], gp, h->st);
        rc = export_impl<float>(h, jet, field, out, N);
    }
    return rc;
}

extern "C" int les_debug_stage_wait(les_handle *h, int max_polls)
{
    if (!h) return LES_ERR_ARG;
    if (h->prec != LES_FP32) return fail(h, LES_ERR_ARG, "staging waits exist in FP32 handles only");
    if (max_polls < -1) return fail(h, LES_ERR_ARG, "max_polls must be >= 0, or -1 for the default");
    h->stage_wait_limit = max_polls;
    if (h->gexec) { // the captured step holds the old launch parameters
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return LES_OK;
}

// ---------------------------------------------------------------------------
// Surface probe
// ---------------------------------------------------------------------------

extern "C" int les_set_fused_tiling(les_handle *h, int ty, int kc)
{
    if (!h) return LES_ERR_ARG;
    if (h->prec != LES_FP32) return fail(h, LES_ERR_ARG, "the fused tiling applies to FP32 handles");
    if ((ty != 8 && ty != 16) || kc < -1) return fail(h, LES_ERR_ARG, "ty must be 8 or 16 and kc >= -1");
    int rc = set_fused_tiling(h, ty, kc);
    if (rc) return rc;
    h->tuned = true;
    h->tune_note = "ty=" + std::to_string(ty) + " kc=" + kc_label(kc) +
                   " (set by the caller)";
    if (h->gexec) { // the captured step holds the old work list
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    return LES_OK;
}

extern "C" int les_probe_surface(les_handle *h, const double *xyz, int npts, int every_n, void *dev_out,
                                 int out_capacity_frames)
{
    if (!h) return LES_ERR_ARG;
    if (npts < 0) return fail(h, LES_ERR_ARG, "npts < 0");
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    if (h->d_cell) cudaFree(h->d_cell);
    if (h->d_wts) cudaFree(h->d_wts);
    h->d_cell = nullptr;
    h->d_wts = nullptr;
    h->probe_npts = 0;
    if (npts == 0) return LES_OK;
    if (!xyz || !dev_out || every_n < 1 || out_capacity_frames < 1)
        return fail(h, LES_ERR_ARG, "probe: null pointer, every_n < 1 or capacity < 1");
    JetHost &J = h->J[0];
    if (!J.product) return fail(h, LES_ERR_ARG, "probe needs a Cartesian-product grid");
    std::vector<int> cell(3 * (size_t)npts);
    std::vector<double> wts(3 * (size_t)npts);
    for (int s = 0; s < npts; ++s) {
        for (int a = 0; a < 3; ++a) {
            double X = xyz[(size_t)a * npts + s];
            const std::vector<double> &ax = J.ax[a];
            int found = -1;
            for (int i = 0; i + 1 < (int)ax.size(); ++i)
                if (X >= ax[i] && X <= ax[i + 1]) {
                    found = i;
                    break;
                }
            if (found < 0) return fail(h, LES_ERR_ARG, "probe point outside the grid");
            cell[3 * s + a] = found;
            wts[3 * s + a] = (X - ax[found]) / (ax[found + 1] - ax[found]);
        }
    }
    CK(cudaMalloc((void **)&h->d_cell, cell.size() * sizeof(int)));
    CK(cudaMalloc((void **)&h->d_wts, wts.size() * sizeof(double)));
    CK(cudaMemcpyAsync(h->d_cell, cell.data(), cell.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->d_wts, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
    long long base = h->step / every_n;
    CK(cudaMemcpyAsync(h->d_probe_base, &base, 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->probe_npts = npts;
    h->probe_every = every_n;
    h->probe_cap = out_capacity_frames;
    h->probe_out = dev_out;
    h->probe_base_level = h->step;
    return LES_OK;
}

extern "C" int les_probe_frames(les_handle *h, int64_t *frames)
{
    if (!h || !frames) return LES_ERR_ARG;
    if (h->probe_npts == 0) {
        *frames = 0;
        return LES_OK;
    }
    *frames = h->step / h->probe_every - h->probe_base_level / h->probe_every;
    return LES_OK;
}

extern "C" int64_t les_last_launch_count(les_handle *h) { return h ? h->last_launches : 0; }

extern "C" const char *les_last_error(les_handle *h) { return h ? h->err.c_str() : g_create_err.c_str(); }

extern "C" int les_bounds_checking(void)
{
#ifdef LES_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

extern "C" int les_bounds_violation(les_handle *h, uint64_t *out)
{
    if (!h || !out) return LES_ERR_ARG;
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, h->d_oob, sizeof(v), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *out = (uint64_t)v;
    return LES_OK;
}

extern "C" const char *les_describe(les_handle *h)
{
    if (!h) return "null handle";
    static thread_local std::string d;
    d = std::string(h->prec == LES_FP64 ? "fp64" : "fp32") + " jets=" + std::to_string(h->njets) +
        " device_bytes=" + std::to_string(h->bytes) + " stage=" +
        (h->prec == LES_FP64 ? std::string("point+grads+iface+update")
                             : std::string(h->sep ? "fused separable " : "fused ") + (h->tuned ? h->tune_note : "ty=" + std::to_string(h->fused_ty) + " (untuned)")) +
        " launches_per_step=" + std::to_string(h->launches_per_step);
    return d.c_str();
}

extern "C" int les_destroy(les_handle *h)
{
    if (!h) return LES_ERR_ARG;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->d_cell) cudaFree(h->d_cell);
    if (h->d_wts) cudaFree(h->d_wts);
    if (h->owns && h->base) cudaFree(h->base);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
    return LES_OK;
}
