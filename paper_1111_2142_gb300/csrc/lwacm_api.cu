// C-ABI implementation (include/lwacm.h): context, validation, workspace
// layout, field transfer, stepping (with captured CUDA graphs) and diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lwacm.h"
#include "launch.h"
#include "lwacm_core.cuh"

using namespace lwacm;

namespace {

// NVTX range around an entry point (a no-op unless a profiler is attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int esize(int storage) { return storage == LWACM_F32 ? 4 : 2; }

}  // namespace

struct lwacm_ctx {
    int Q = 0, D = 0, nx = 0, ny = 0, nz = 0, bc = 0, nf = 0;
    double nu = 0, nu_p = 0;  // nu_p: viscosity of the pressure update (0: nu)
    double alpha = 0;         // diffusivity of the passive scalar (0: no scalar)
    double gamma = 0;         // D2Q9 bulk-viscosity variant (Appendix "Computing derivatives locally")
    bool bulk = false;        // the variant is on: Tr+ - Tr^(e) is the field after the flow fields
    bool semi = false;        // semi-implicit pressure update (Eq. FDcompact_si)
    bool sr = false;          // BF16 / FP16 stores rounded stochastically (half-row kernel)
    bool scalar_rows = false; // the passive scalar on its own row-tiled kernel after the flow kernel
    int nsc = 0;              // fields stored after the flow fields: the scalar or the trace (0 or 1)
    long long N = 0, Nal = 0;
    double lid[3] = {0, 0, 0}, force[3] = {0, 0, 0}, rho0 = 1.0;
    int storage = LWACM_F32;
    int graph_chunk = 64;
    int kernel_opt = 0;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t off_buf[2] = {0, 0}, off_stage = 0, off_partial = 0, off_diag = 0, off_err = 0, total = 0;
    // per-node force field (LWACM_OPT_FORCE_FIELD): D FP32 fields in the workspace
    bool ff_reserved = false, ff_active = false;
    size_t off_ff = 0;
    cudaStream_t stream = nullptr;
    bool bound = false, has_fields = false;
    int cur = 0;
    long long steps = 0;
    // status
    lwacm_status sticky = LWACM_OK;
    std::string err;
    // graphs: one per starting buffer parity
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gchunk[2] = {0, 0};
    int kernel = 1;  // 1 generic, 4 batch, 5 half-row TMA, 6 D2Q9 2D tiles (2 and 3: retired
                     // row-tiled kernels, superseded by 5)
    std::string kname = "none";
    // batched domains (nbatch > 0): packed one after the other
    int nbatch = 0;
    std::vector<BatchDomain> doms;
    std::vector<BatchTile> tiles;    // 1D tiles (shape 0)
    std::vector<BatchTile2> tiles2;  // 2D tiles of the current shape (shape > 0)
    int batch_shape = 0;
    size_t tiles_cap = 0;  // table entries reserved in the workspace (largest over the shapes)
    size_t off_doms = 0, off_tiles = 0, off_bar = 0;
    int batch_mode = 0;  // 0: one launch per step (graphs), 1: one persistent launch
    long long withhold = -1;
    // recorded forward run for lwacm_backward
    char *adj = nullptr;
    size_t adj_bytes = 0;
    long long rec_T = -1;
    int rec_S = 0;
    bool rec_last_kept = false;  // the last segment's states are in the segment buffer
};

namespace {

lwacm_status fail(lwacm_ctx *c, lwacm_status s, const std::string &msg) {
    if (c) {
        c->err = msg;
        if (s == LWACM_E_CUDA || s == LWACM_E_TIMEOUT) c->sticky = s;
    }
    return s;
}

lwacm_status cuda_fail(lwacm_ctx *c, cudaError_t e, const char *where) {
    return fail(c, LWACM_E_CUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                                     cudaGetErrorString(e) + ")");
}

#define CK(ctx, call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

void layout(lwacm_ctx *c) {
    const size_t fbytes = (size_t)c->Nal * esize(c->storage);
    size_t off = 0;
    for (int b = 0; b < 2; ++b) {
        c->off_buf[b] = off;
        off = align_up(off + fbytes * (c->nf + c->nsc), kAlign);
    }
    c->off_stage = off;
    off = align_up(off + (size_t)c->Nal * 8, kAlign);
    c->off_partial = off;
    off = align_up(off + (size_t)kDiagBlocks * kDiagValues * 8, kAlign);
    c->off_diag = off;
    off = align_up(off + 16 * 8, kAlign);
    c->off_err = off;
    off = align_up(off + 16, kAlign);
    if (c->ff_reserved) {
        c->off_ff = off;
        off = align_up(off + (size_t)c->Nal * 4 * c->D, kAlign);
    }
    if (c->nbatch) {
        c->off_doms = off;
        off = align_up(off + sizeof(BatchDomain) * c->doms.size(), kAlign);
        c->off_tiles = off;
        off = align_up(off + 16 * c->tiles_cap, kAlign);
        c->off_bar = off;
        off = align_up(off + 16, kAlign);
    }
    c->total = off;
}

StepParams params(const lwacm_ctx *c) {
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.nx = c->nx;
    p.ny = c->ny;
    p.nz = c->nz;
    p.bc = c->bc;
    p.N = c->N;
    p.fstride = c->Nal;
    // Eq. viscosity2 / Eq. ACM2.0nu: a = 2(omega-1)/omega = 1 - 6 nu; s = 3(1-a) = 18 nu
    p.s = (float)(18.0 * c->nu);
    p.a = (float)(1.0 - 6.0 * c->nu);
    p.am1 = (float)(-6.0 * c->nu);
    // Eq. ACM2.0ccccbb: (2/omega - 1) * 2 f^(e,o)(rho0, u_w) = 6 nu * 2 * 3 w rho0 (c.u_w)
    p.wallc = (float)(36.0 * c->nu * c->rho0);
    for (int a = 0; a < 3; ++a) {
        p.lid[a] = (float)c->lid[a];
        p.force[a] = (float)c->force[a];
    }
    p.has_force = (c->force[0] != 0 || c->force[1] != 0 || c->force[2] != 0) ? 1 : 0;
    p.gfield = (c->ff_active && c->ws) ? (const float *)(c->ws + c->off_ff) : nullptr;
    p.sdelta = c->nu_p > 0 ? (float)(18.0 * (c->nu_p - c->nu)) : 0.f;
    p.scalar = c->alpha != 0 ? 1 : 0;
    p.at = (float)(1.0 - 6.0 * c->alpha);  // a_t = 2(omega_t - 1)/omega_t, alpha = (1/omega_t - 1/2)/3
    p.bulk = c->bulk ? 1 : 0;
    p.gamma = (float)c->gamma;
    p.err = c->ws ? (int *)(c->ws + c->off_err) : nullptr;
    // the stochastic-rounding step counter: the word after the error word
    p.sr_ctr = c->sr && c->ws ? (unsigned *)(c->ws + c->off_err) + 1 : nullptr;
    // omega_p on the half-row kernel: the staging buffer (unused during steps) holds
    // the density term k_nup_sum forms before each step
    p.nup_p = p.sdelta != 0.f && c->ws ? (float *)(c->ws + c->off_stage) : nullptr;
    p.walled[0] = p.walled[1] = p.walled[2] = 0;
    p.lid_axis = c->D - 1;
    if (c->bc == LWACM_BC_CAVITY) {
        for (int a = 0; a < c->D; ++a) p.walled[a] = 1;
    } else if (c->bc == LWACM_BC_CHANNEL) {
        p.walled[1] = 1;
        p.lid_axis = 1;
    }
    return p;
}

void drop_graphs(lwacm_ctx *c) {
    for (int k = 0; k < 2; ++k) {
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        c->gexec[k] = nullptr;
        c->gchunk[k] = 0;
    }
}

// Interior kernel: the explicit choice if it supports the shape, else (automatic)
// the half-row TMA kernel (D3Q19), then the 2D-tile kernel (D2Q9), then the
// generic gather kernel, which supports everything. Returns false when an
// explicit choice is not supported. Kernels that need the device are only
// considered once a workspace is bound.
bool choose_kernel(lwacm_ctx *c) {
    if (c->nbatch) {
        c->kernel = 4;
        static const char *names[2][8] = {
            {"batch_step", "batch_tiles30x6_step", "batch_tiles30x14_step", "batch_tiles62x6_step",
             "batch_tiles30x30_step", "batch_tiles62x14_step", "batch_tiles126x6_step", "batch_step"},
            {"batch_persistent", "batch_tiles30x6_persistent", "batch_tiles30x14_persistent",
             "batch_tiles62x6_persistent", "batch_tiles30x30_persistent", "batch_tiles62x14_persistent",
             "batch_tiles126x6_persistent", "batch_persistent"}};
        c->kname = names[c->batch_mode ? 1 : 0][c->batch_shape & 7];
        return c->kernel_opt == 0 || c->kernel_opt == 1;
    }
    const StepParams p = params(c);
    const bool dev = c->bound;
    // the passive scalar: on its own row-tiled kernel when the shape allows, the
    // flow then on the half-row kernel; otherwise both on the generic kernel
    c->scalar_rows = dev && p.scalar && scalar_rows_supported(c->Q, c->storage, p);
    StepParams pf = p;
    if (c->scalar_rows) pf.scalar = 0;
    const bool h_ok = dev && half_supported(c->Q, c->storage, pf);
    const bool s_ok = tiles2d_supported(c->Q, c->storage, p);
    bool ok = true;
    if (c->sr) {  // only the half-row kernel rounds stochastically: no fallback
        c->kernel = h_ok ? 5 : 1;
        ok = (c->kernel_opt == 0 || c->kernel_opt == 5) && (h_ok || !dev);
    } else switch (c->kernel_opt) {
        case 1: c->kernel = 1; break;
        case 5: c->kernel = h_ok ? 5 : 1; ok = h_ok || !dev; break;
        case 6: c->kernel = s_ok ? 6 : 1; ok = s_ok; break;
        default: c->kernel = h_ok ? 5 : (s_ok ? 6 : 1); break;
    }
    static const char *gname[2] = {"generic_d2q9", "generic_d3q19"};
    static const char *sname[7] = {"tiles2d_d2q9_30x14", "tiles2d_d2q9_30x6",  "tiles2d_d2q9_30x14", "tiles2d_d2q9_62x6",
                                   "tiles2d_d2q9_30x30", "tiles2d_d2q9_62x14", "tiles2d_d2q9_126x6"};
    if (c->kernel != 5) c->scalar_rows = false;
    static const char *hname[2][2] = {{"half_d3q19_tma", "half_d3q19_tma+scalar_rows"},
                                      {"half_d3q19_tma+nu_p_sum", "half_d3q19_tma+nu_p_sum+scalar_rows"}};
    c->kname = c->kernel == 5   ? hname[p.sdelta != 0.f ? 1 : 0][c->scalar_rows ? 1 : 0]
               : c->kernel == 6 ? sname[c->batch_shape >= 0 && c->batch_shape < 7 ? c->batch_shape : 0]
                                : gname[c->Q == 19 ? 1 : 0];
    return ok;
}

void *bufp(lwacm_ctx *c, int b) { return c->ws + c->off_buf[b]; }

size_t field_bytes(const lwacm_ctx *c) { return (size_t)c->Nal * esize(c->storage); }

// 2D tiles of shape k over every domain (D2Q9): row-major within a domain
void build_tiles2(const lwacm_ctx *c, int k, std::vector<BatchTile2> &out) {
    out.clear();
    int tw = 0, th = 0;
    batch_shape(k, &tw, &th);
    for (int b = 0; b < c->nbatch; ++b)
        for (int y = 0; y < c->doms[b].ny; y += th)
            for (int x = 0; x < c->doms[b].nx; x += tw) out.push_back(BatchTile2{b, x, y, 0});
}

// upload the tile table of the current shape (host tables are pageable: synchronise)
lwacm_status upload_tiles(lwacm_ctx *c) {
    if (c->batch_shape > 0) {
        build_tiles2(c, c->batch_shape, c->tiles2);
        CK(c, cudaMemcpyAsync(c->ws + c->off_tiles, c->tiles2.data(), sizeof(BatchTile2) * c->tiles2.size(),
                              cudaMemcpyHostToDevice, c->stream),
           "tile table");
    } else {
        CK(c, cudaMemcpyAsync(c->ws + c->off_tiles, c->tiles.data(), sizeof(BatchTile) * c->tiles.size(),
                              cudaMemcpyHostToDevice, c->stream),
           "tile table");
    }
    CK(c, cudaStreamSynchronize(c->stream), "sync");
    return LWACM_OK;
}

BatchParams batch_params(lwacm_ctx *c) {
    BatchParams bp;
    bp.doms = (const BatchDomain *)(c->ws + c->off_doms);
    bp.tiles = (const BatchTile *)(c->ws + c->off_tiles);
    bp.tiles2 = (const BatchTile2 *)(c->ws + c->off_tiles);
    bp.shape = c->batch_shape;
    bp.ntiles = (long long)(c->batch_shape > 0 ? c->tiles2.size() : c->tiles.size());
    bp.fstride = c->Nal;
    bp.bar_count = (unsigned *)(c->ws + c->off_bar);
    bp.bar_gen = bp.bar_count + 1;
    bp.err = (int *)(c->ws + c->off_err);
    bp.withhold_step = c->withhold;
    return bp;
}

// enqueue one time step from state `in` to state `out` (each nf fields x Nal)
cudaError_t step_between(lwacm_ctx *c, const void *in, void *out, cudaStream_t st) {
    if (c->nbatch) return launch_batch_step(c->Q, c->storage, in, out, batch_params(c), st);
    const StepParams p = params(c);
    StepParams pf = p;
    if (c->scalar_rows) pf.scalar = 0;  // the flow kernel leaves the scalar to its own kernel
    cudaError_t e = cudaSuccess;
    if (c->kernel == 5 && p.sdelta != 0.f) e = launch_nup_sum(c->storage, in, p.nup_p, p, st);
    if (e != cudaSuccess) return e;
    e = c->kernel == 5               ? launch_step_half(c->Q, c->storage, in, out, pf, st)
                    : c->kernel == 6 ? launch_step_tiles2d(c->Q, c->storage, c->batch_shape > 0 ? c->batch_shape : 2,
                                                           in, out, p, st)
                                     : launch_step_generic(c->Q, c->storage, in, out, p, st);
    if (e != cudaSuccess) return e;
    // the 2D-tile kernel applies the wall rule itself; the half-row kernel the x-face
    // walls of a cavity whose lid is not on an x face
    if (c->bc != LWACM_BC_PERIODIC && c->kernel != 6) {
        StepParams pw = p;
        pw.xfaces_done = c->kernel == 5 && half_xwalls(p) ? 1 : 0;
        e = launch_wall_pass(c->Q, c->storage, in, out, pw, st);
    }
    if (e == cudaSuccess && p.sr_ctr && c->kernel == 5) e = launch_sr_tick(p.sr_ctr, st);
    if (e == cudaSuccess && c->semi) e = launch_semi_implicit(c->Q, c->storage, in, out, p, st);
    if (e == cudaSuccess && c->scalar_rows) e = launch_scalar_rows(in, out, p, st);
    return e;
}

// enqueue one time step: buffer cur -> buffer 1-cur
cudaError_t enqueue_step(lwacm_ctx *c, int cur, cudaStream_t st) {
    return step_between(c, bufp(c, cur), bufp(c, 1 - cur), st);
}

// adjoint workspace: K checkpoints, S+1 segment states, 2 lambda / (Dbar, Jbar)
// states, one more (Dbar, Jbar) state, dL/dnu partials, total and block counter
struct AdjLayout {
    long long K = 0;
    int S = 0;
    size_t state = 0, ckpt = 0, seg = 0, lam = 0, dj = 0, part = 0, total = 0, bytes = 0;
};
AdjLayout adj_layout(const lwacm_ctx *c, long long T, int stride) {
    AdjLayout L;
    L.S = stride > 0 ? stride : (int)std::ceil(std::sqrt((double)(T > 0 ? T : 1)));
    L.K = T > 0 ? (T + L.S - 1) / L.S : 1;
    L.state = align_up((size_t)c->Nal * 4 * c->nf, kAlign);
    size_t off = 0;
    L.ckpt = off;
    off += L.state * (size_t)L.K;
    L.seg = off;
    off += L.state * (size_t)(L.S + 1);
    L.lam = off;
    off += L.state * 2;
    L.dj = off;
    off += L.state;
    L.part = off;
    off = align_up(off + (size_t)adjoint_partials() * 8, kAlign);
    L.total = off;
    off = align_up(off + 64, kAlign);
    L.bytes = off;
    return L;
}

lwacm_status ready(lwacm_ctx *c, bool need_fields) {
    if (!c) return LWACM_E_ARG;
    if (c->sticky != LWACM_OK) return c->sticky;
    if (!c->bound) return fail(c, LWACM_E_STATE, "no workspace bound (call lwacm_bind)");
    if (need_fields && !c->has_fields)
        return fail(c, LWACM_E_STATE, "fields not initialised (call lwacm_set_fields)");
    return LWACM_OK;
}

lwacm_status build_graph(lwacm_ctx *c, int parity, int chunk) {
    if (!c->cap_stream) CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream create");
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int cur = parity;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < chunk && le == cudaSuccess; ++k) {
        le = enqueue_step(c, cur, c->cap_stream);
        cur ^= 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, le, "capture launch");
    }
    if (ee != cudaSuccess) return cuda_fail(c, ee, "end capture");
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(c, ie, "graph instantiate");
    c->gexec[parity] = ex;
    c->gchunk[parity] = chunk;
    return LWACM_OK;
}

// ---- autotuner helpers --------------------------------------------------------
struct Cand {
    int kernel, tile, mode;
};

// FNV-1a over the bytes of v
void fnv(uint64_t &h, const void *v, size_t n) {
    const unsigned char *p = (const unsigned char *)v;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
}

// problem key: lattice, storage, boundary, shape (or the ensemble's sizes and
// viscosities, hashed), forcing, and the device (SM count, compute capability)
std::string tune_key(const lwacm_ctx *c) {
    int dev = 0, sms = 0, mj = 0, mn = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&mj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mn, cudaDevAttrComputeCapabilityMinor, dev);
    char buf[256];
    if (c->nbatch) {
        uint64_t h = 1469598103934665603ULL;
        for (const BatchDomain &d : c->doms) {
            fnv(h, &d.nx, sizeof d.nx);
            fnv(h, &d.ny, sizeof d.ny);
            fnv(h, &d.nz, sizeof d.nz);
            fnv(h, &d.s, sizeof d.s);
        }
        std::snprintf(buf, sizeof buf, "lattice=%d;storage=%d;batch=%d;nodes=%lld;domains=%016llx;sm=%d;cc=%d.%d",
                      c->Q, c->storage, c->nbatch, c->N, (unsigned long long)h, sms, mj, mn);
    } else {
        const bool forced = c->force[0] != 0 || c->force[1] != 0 || c->force[2] != 0 || c->ff_active;
        std::snprintf(buf, sizeof buf, "lattice=%d;storage=%d;bc=%d;nx=%d;ny=%d;nz=%d;force=%d;sm=%d;cc=%d.%d", c->Q,
                      c->storage, c->bc, c->nx, c->ny, c->nz, forced ? 1 : 0, sms, mj, mn);
    }
    return buf;
}

std::vector<Cand> tune_candidates(const lwacm_ctx *c) {
    std::vector<Cand> v;
    if (c->nbatch) {
        for (int k = 0; k < batch_shapes(); ++k)
            if (batch_shape_supported(c->Q, c->storage, k))
                for (int m = 0; m < 2; ++m) v.push_back(Cand{0, k, m});
    } else {
        const int ks[2] = {5, 1};
        for (int k : ks) v.push_back(Cand{k, 0, 0});
        if (c->Q == 9)
            for (int k = 1; k < batch_shapes(); ++k) v.push_back(Cand{6, k, 0});
    }
    return v;
}

lwacm_status apply_cand(lwacm_ctx *c, const Cand &k) {
    if (c->nbatch) {
        lwacm_status s = lwacm_set_option(c, LWACM_OPT_BATCH_TILE, k.tile);
        if (s == LWACM_OK) s = lwacm_set_option(c, LWACM_OPT_BATCH_MODE, k.mode);
        return s;
    }
    if (k.kernel == 6) {
        const lwacm_status s = lwacm_set_option(c, LWACM_OPT_BATCH_TILE, k.tile);
        if (s != LWACM_OK) return s;
    }
    const lwacm_status s = lwacm_set_option(c, LWACM_OPT_KERNEL, k.kernel);
    if (s != LWACM_OK) return s;
    return c->kernel == k.kernel ? LWACM_OK : LWACM_E_UNSUPPORTED;
}

// the rest state (all fields zero) in buffer 0, marked as set
lwacm_status tune_zero_state(lwacm_ctx *c) {
    CK(c, cudaMemsetAsync(bufp(c, 0), 0, field_bytes(c) * (c->nf + c->nsc), c->stream), "zero state");
    c->cur = 0;
    c->has_fields = true;
    c->steps = 0;
    return LWACM_OK;
}

}  // namespace

extern "C" {

lwacm_status lwacm_create(int lattice, int nx, int ny, int nz, double nu, int bc,
                          lwacm_ctx **out) {
    if (!out) return LWACM_E_ARG;
    *out = nullptr;
    if (lattice != LWACM_D2Q9 && lattice != LWACM_D3Q19) return LWACM_E_ARG;
    if (bc != LWACM_BC_PERIODIC && bc != LWACM_BC_CAVITY && bc != LWACM_BC_CHANNEL)
        return LWACM_E_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return LWACM_E_ARG;
    if (lattice == LWACM_D2Q9 && nz != 1) return LWACM_E_ARG;
    if (bc == LWACM_BC_CAVITY && (nx < 2 || ny < 2 || (lattice == LWACM_D3Q19 && nz < 2)))
        return LWACM_E_ARG;
    if (bc == LWACM_BC_CHANNEL && ny < 2) return LWACM_E_ARG;
    if ((long long)nx * ny * nz > (1LL << 40)) return LWACM_E_ARG;
    // Section 2.3: stable for 1 <= omega < 2, i.e. 0 < nu <= 1/6 (Eq. viscosity2)
    if (!(nu > 0.0) || !(nu <= 1.0 / 6.0 + 1e-15) || !std::isfinite(nu)) return LWACM_E_RANGE;
    lwacm_ctx *c = new (std::nothrow) lwacm_ctx();
    if (!c) return LWACM_E_NOMEM;
    c->Q = lattice;
    c->D = lattice == LWACM_D2Q9 ? 2 : 3;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->bc = bc;
    c->nu = nu;
    c->nf = c->D + 1;
    c->N = (long long)nx * ny * nz;
    c->Nal = (long long)align_up((size_t)c->N, 64);
    layout(c);
    choose_kernel(c);
    *out = c;
    return LWACM_OK;
}

lwacm_status lwacm_batch_create(int lattice, int n, const int *nx, const int *ny, const int *nz,
                                const double *nu, int bc, lwacm_ctx **out) {
    if (!out) return LWACM_E_ARG;
    *out = nullptr;
    if (n < 1 || !nx || !ny || !nu) return LWACM_E_ARG;
    if (lattice != LWACM_D2Q9 && lattice != LWACM_D3Q19) return LWACM_E_ARG;
    if (lattice == LWACM_D3Q19 && !nz) return LWACM_E_ARG;
    if (bc != LWACM_BC_PERIODIC) return LWACM_E_UNSUPPORTED;
    lwacm_ctx *c = new (std::nothrow) lwacm_ctx();
    if (!c) return LWACM_E_NOMEM;
    c->Q = lattice;
    c->D = lattice == LWACM_D2Q9 ? 2 : 3;
    c->nf = c->D + 1;
    c->bc = bc;
    c->nbatch = n;
    long long off = 0;
    const int tile = batch_tile();
    try {
        c->doms.resize(n);
        for (int b = 0; b < n; ++b) {
            const int z = lattice == LWACM_D2Q9 ? 1 : nz[b];
            if (nx[b] < 1 || ny[b] < 1 || z < 1 || (lattice == LWACM_D2Q9 && nz && nz[b] != 1)) {
                delete c;
                return LWACM_E_ARG;
            }
            if (!(nu[b] > 0.0) || !(nu[b] <= 1.0 / 6.0 + 1e-15) || !std::isfinite(nu[b])) {
                delete c;
                return LWACM_E_RANGE;
            }
            BatchDomain &d = c->doms[b];
            d.nx = nx[b];
            d.ny = ny[b];
            d.nz = z;
            d.pad = 0;
            d.off = off;
            d.n = (long long)nx[b] * ny[b] * z;
            d.s = (float)(18.0 * nu[b]);  // Eq. ACM2.0nu: s = 18 nu, a = 1 - 6 nu
            d.a = (float)(1.0 - 6.0 * nu[b]);
            for (long long t = 0; t < d.n; t += tile) {
                BatchTile bt;
                bt.dom = b;
                bt.pad = 0;
                bt.start = off + t;
                c->tiles.push_back(bt);
            }
            off += d.n;
        }
    } catch (...) {
        delete c;
        return LWACM_E_NOMEM;
    }
    try {
        c->tiles_cap = c->tiles.size();
        if (lattice == LWACM_D2Q9) {
            std::vector<BatchTile2> t2;
            for (int k = 1; k < batch_shapes(); ++k) {
                build_tiles2(c, k, t2);
                c->tiles_cap = std::max(c->tiles_cap, t2.size());
            }
        }
    } catch (...) {
        delete c;
        return LWACM_E_NOMEM;
    }
    c->nu = nu[0];
    c->nx = (int)std::min<long long>(off, 1LL << 30);
    c->ny = 1;
    c->nz = 1;
    c->N = off;
    c->Nal = (long long)align_up((size_t)c->N, 64);
    layout(c);
    choose_kernel(c);
    *out = c;
    return LWACM_OK;
}

lwacm_status lwacm_batch_offsets(const lwacm_ctx *c, long long *offsets) {
    if (!c || !offsets) return LWACM_E_ARG;
    if (!c->nbatch) {
        offsets[0] = 0;
        offsets[1] = c->N;
        return LWACM_OK;
    }
    for (int b = 0; b < c->nbatch; ++b) offsets[b] = c->doms[b].off;
    offsets[c->nbatch] = c->N;
    return LWACM_OK;
}

lwacm_status lwacm_set_option(lwacm_ctx *c, int key, double v) {
    if (!c) return LWACM_E_ARG;
    if (c->sticky != LWACM_OK) return c->sticky;
    if (!std::isfinite(v)) return fail(c, LWACM_E_ARG, "non-finite option value");
    switch (key) {
        case LWACM_OPT_LID_X: case LWACM_OPT_LID_Y: case LWACM_OPT_LID_Z:
            c->lid[key - LWACM_OPT_LID_X] = v;
            break;
        case LWACM_OPT_FORCE_X: case LWACM_OPT_FORCE_Y: case LWACM_OPT_FORCE_Z:
            c->force[key - LWACM_OPT_FORCE_X] = v;
            break;
        case LWACM_OPT_RHO0:
            if (!(v > 0)) return fail(c, LWACM_E_ARG, "rho0 must be > 0");
            c->rho0 = v;
            break;
        case LWACM_OPT_STORAGE: {
            const int s = (int)v;
            if (s != LWACM_F32 && s != LWACM_BF16 && s != LWACM_F16)
                return fail(c, LWACM_E_ARG, "storage must be F32, BF16 or F16");
            if (c->bound) return fail(c, LWACM_E_STATE, "storage type is fixed once bound");
            if (s == LWACM_F32 && c->sr) return fail(c, LWACM_E_UNSUPPORTED, "stochastic rounding needs BF16 or FP16 storage");
            c->storage = s;
            layout(c);
            break;
        }
        case LWACM_OPT_GRAPH_CHUNK: {
            const int g = (int)v;
            if (g < 0 || (g & 1) || g > 100000)
                return fail(c, LWACM_E_ARG, "graph chunk must be even, >= 0");
            c->graph_chunk = g;
            break;
        }
        case LWACM_OPT_KERNEL: {
            const int k = (int)v;
            if (k < 0 || k > 6 || k == 4 || k == 2 || k == 3)
                return fail(c, LWACM_E_ARG, "kernel must be 0, 1, 5 or 6");
            const int old = c->kernel_opt;
            c->kernel_opt = k;
            if (!choose_kernel(c)) {
                c->kernel_opt = old;
                choose_kernel(c);
                return fail(c, LWACM_E_UNSUPPORTED, "this kernel does not support the shape/boundary/storage");
            }
            break;
        }
        case LWACM_OPT_BATCH_MODE: {
            const int m = (int)v;
            if (m != 0 && m != 1) return fail(c, LWACM_E_ARG, "batch mode must be 0 or 1");
            if (!c->nbatch) return fail(c, LWACM_E_STATE, "not a batched context");
            c->batch_mode = m;
            break;
        }
        case LWACM_OPT_SCALAR_ALPHA: {
            if (c->nbatch) return fail(c, LWACM_E_UNSUPPORTED, "no scalar in batched contexts");
            if (c->bound) return fail(c, LWACM_E_STATE, "the scalar is set up before lwacm_bind");
            if (v != 0 && !(v > 0.0 && v <= 1.0 / 6.0 + 1e-15))
                return fail(c, LWACM_E_RANGE, "alpha must be in (0, 1/6] (or 0: no scalar)");
            if (v != 0 && c->bc != LWACM_BC_PERIODIC)
                return fail(c, LWACM_E_UNSUPPORTED, "the scalar is for periodic domains");
            if (v != 0 && c->bulk) return fail(c, LWACM_E_UNSUPPORTED, "not with the bulk-viscosity variant");
            if (v != 0 && c->semi) return fail(c, LWACM_E_UNSUPPORTED, "not with the semi-implicit pressure update");
            c->alpha = v;
            c->nsc = v != 0 ? 1 : 0;
            layout(c);
            break;
        }
        case LWACM_OPT_BULK_GAMMA: {
            if (c->nbatch) return fail(c, LWACM_E_UNSUPPORTED, "no bulk-viscosity variant in batched contexts");
            if (c->bound) return fail(c, LWACM_E_STATE, "the bulk-viscosity variant is set up before lwacm_bind");
            if (!(v > -1.0 && v < 1.0)) return fail(c, LWACM_E_RANGE, "gamma must be in (-1, 1)");
            if (v != 0 && (c->Q != 9 || c->bc != LWACM_BC_PERIODIC))
                return fail(c, LWACM_E_UNSUPPORTED, "the bulk-viscosity variant is for periodic D2Q9 domains");
            if (v != 0 && c->alpha != 0) return fail(c, LWACM_E_UNSUPPORTED, "not with the passive scalar");
            if (v != 0 && c->semi) return fail(c, LWACM_E_UNSUPPORTED, "not with the semi-implicit pressure update");
            c->gamma = v;
            c->bulk = v != 0;
            c->nsc = c->bulk ? 1 : 0;
            layout(c);
            break;
        }
        case LWACM_OPT_STOCHASTIC_ROUNDING: {
            if (v != 0 && v != 1) return fail(c, LWACM_E_ARG, "stochastic rounding must be 0 or 1");
            if (v != 0 && (c->nbatch || c->Q != 19 || c->bc != LWACM_BC_PERIODIC))
                return fail(c, LWACM_E_UNSUPPORTED, "stochastic rounding is for single periodic D3Q19 domains");
            if (v != 0 && c->storage == LWACM_F32)
                return fail(c, LWACM_E_UNSUPPORTED, "stochastic rounding needs BF16 or FP16 storage");
            if (v != 0 && (c->semi || c->alpha != 0 || c->bulk || c->nu_p > 0 || c->ff_reserved))
                return fail(c, LWACM_E_UNSUPPORTED, "stochastic rounding is for the plain scheme");
            c->sr = v != 0;
            drop_graphs(c);
            break;
        }
        case LWACM_OPT_SEMI_IMPLICIT: {
            if (v != 0 && v != 1) return fail(c, LWACM_E_ARG, "semi-implicit must be 0 or 1");
            if (v != 0 && (c->nbatch || c->bc != LWACM_BC_PERIODIC))
                return fail(c, LWACM_E_UNSUPPORTED, "the semi-implicit pressure update is for single periodic domains");
            if (v != 0 && (c->alpha != 0 || c->bulk))
                return fail(c, LWACM_E_UNSUPPORTED, "not with the passive scalar or the bulk-viscosity variant");
            c->semi = v != 0;
            drop_graphs(c);
            break;
        }
        case LWACM_OPT_NU_P: {
            if (c->nbatch) return fail(c, LWACM_E_UNSUPPORTED, "no omega_p in batched contexts");
            if (v != 0 && !(v > 0.0 && v <= 1.0 / 6.0 + 1e-15))
                return fail(c, LWACM_E_RANGE, "nu_p must be in (0, 1/6] (or 0: same as nu)");
            if (v != 0 && c->bc != LWACM_BC_PERIODIC)
                return fail(c, LWACM_E_UNSUPPORTED, "omega_p is for periodic domains");
            c->nu_p = v;
            break;
        }
        case LWACM_OPT_BATCH_TILE: {
            const int k = (int)v;
            if (k < 0 || k >= batch_shapes() || (double)k != v) return fail(c, LWACM_E_ARG, "unknown tile shape");
            if (!batch_shape_supported(c->Q, c->storage, k))
                return fail(c, LWACM_E_UNSUPPORTED, "2D tile shapes are for the D2Q9 lattice");
            c->batch_shape = k;
            if (c->bound && c->nbatch) {
                const lwacm_status ts = upload_tiles(c);
                if (ts != LWACM_OK) return ts;
            }
            break;
        }
        case LWACM_OPT_FORCE_FIELD: {
            const int r = (int)v;
            if (r != 0 && r != 1) return fail(c, LWACM_E_ARG, "force field option must be 0 or 1");
            if (c->nbatch) return fail(c, LWACM_E_UNSUPPORTED, "no force field in batched contexts");
            if (c->bound) return fail(c, LWACM_E_STATE, "the force field is reserved before lwacm_bind");
            c->ff_reserved = r != 0;
            c->ff_active = false;
            layout(c);
            break;
        }
        case LWACM_OPT_TEST_WITHHOLD:
            if (!c->nbatch) return fail(c, LWACM_E_STATE, "not a batched context");
            c->withhold = (long long)v;
            break;
        default:
            return fail(c, LWACM_E_ARG, "unknown option key");
    }
    choose_kernel(c);
    drop_graphs(c);
    return LWACM_OK;
}

lwacm_status lwacm_workspace_bytes(const lwacm_ctx *c, size_t *bytes) {
    if (!c || !bytes) return LWACM_E_ARG;
    *bytes = c->total;
    return LWACM_OK;
}

lwacm_status lwacm_bind(lwacm_ctx *c, void *ws, size_t bytes, void *stream) {
    if (!c) return LWACM_E_ARG;
    if (c->sticky != LWACM_OK) return c->sticky;
    if (!ws) return fail(c, LWACM_E_ARG, "null workspace");
    if (((uintptr_t)ws) % kAlign) return fail(c, LWACM_E_ARG, "workspace not 256-byte aligned");
    if (bytes < c->total) return fail(c, LWACM_E_NOMEM, "workspace smaller than lwacm_workspace_bytes");
    drop_graphs(c);
    c->ws = (char *)ws;
    c->ws_bytes = bytes;
    c->stream = (cudaStream_t)stream;
    c->bound = true;
    c->has_fields = false;
    c->cur = 0;
    c->steps = 0;
    CK(c, cudaMemsetAsync(c->ws + c->off_err, 0, 16, c->stream), "clear error word");
    if (c->nbatch) {
        CK(c, cudaMemcpyAsync(c->ws + c->off_doms, c->doms.data(), sizeof(BatchDomain) * c->doms.size(),
                              cudaMemcpyHostToDevice, c->stream),
           "domain table");
        CK(c, cudaStreamSynchronize(c->stream), "sync");  // the host tables are pageable
        const lwacm_status ts = upload_tiles(c);
        if (ts != LWACM_OK) return ts;
    }
    if (!choose_kernel(c)) {
        c->kernel_opt = 0;
        choose_kernel(c);
        return fail(c, LWACM_E_UNSUPPORTED, "the requested kernel does not support the shape/boundary/storage");
    }
    return LWACM_OK;
}

lwacm_status lwacm_set_fields(lwacm_ctx *c, const void *d, const void *ux, const void *uy,
                              const void *uz, int dtype, int where) {
    const Range range("lwacm_set_fields");
    lwacm_status s = ready(c, false);
    if (s != LWACM_OK) return s;
    if (!d || !ux || !uy || (c->Q == 19 && !uz) || (c->Q == 9 && uz))
        return fail(c, LWACM_E_ARG, "field pointers: d, ux, uy required; uz iff D3Q19");
    if (dtype != LWACM_F32 && dtype != LWACM_F64) return fail(c, LWACM_E_ARG, "dtype must be F32 or F64");
    if (where != LWACM_DEVICE && where != LWACM_HOST) return fail(c, LWACM_E_ARG, "bad location");
    const void *src[4] = {d, ux, uy, uz};
    const size_t sb = dtype == LWACM_F64 ? 8 : 4;
    const size_t nbytes = (size_t)c->N * sb;
    c->cur = 0;
    char *dst = (char *)bufp(c, 0);
    for (int f = 0; f < c->nf; ++f) {
        char *fd = dst + (size_t)f * field_bytes(c);
        if (where == LWACM_HOST && dtype == LWACM_F32 && c->storage == LWACM_F32) {
            CK(c, cudaMemcpyAsync(fd, src[f], nbytes, cudaMemcpyHostToDevice, c->stream), "H2D");
            continue;
        }
        const void *dsrc = src[f];
        if (where == LWACM_HOST) {
            CK(c, cudaMemcpyAsync(c->ws + c->off_stage, src[f], nbytes, cudaMemcpyHostToDevice, c->stream),
               "H2D stage");
            dsrc = c->ws + c->off_stage;
        }
        CK(c, launch_convert_in(c->storage, dtype, dsrc, fd, c->N, c->stream), "convert in");
    }
    // the scalar starts at zero until lwacm_set_scalar; the trace deviation of the
    // bulk-viscosity variant at zero (Tr^(+) = Tr^(e): the first step is the standard one)
    if (c->nsc) CK(c, cudaMemsetAsync(dst + (size_t)c->nf * field_bytes(c), 0, field_bytes(c), c->stream), "zero extra");
    c->has_fields = true;
    c->steps = 0;
    return LWACM_OK;
}

lwacm_status lwacm_set_force_field(lwacm_ctx *c, const void *gx, const void *gy, const void *gz, int dtype,
                                   int where) {
    lwacm_status s = ready(c, false);
    if (s != LWACM_OK) return s;
    if (!c->ff_reserved) return fail(c, LWACM_E_STATE, "no force field reserved (LWACM_OPT_FORCE_FIELD before bind)");
    if (!gx && !gy && !gz) {
        if (c->ff_active) {
            c->ff_active = false;
            choose_kernel(c);
            drop_graphs(c);
        }
        return LWACM_OK;
    }
    if (!gx || !gy || (c->Q == 19 && !gz) || (c->Q == 9 && gz))
        return fail(c, LWACM_E_ARG, "force field pointers: gx, gy required; gz iff D3Q19");
    if (dtype != LWACM_F32 && dtype != LWACM_F64) return fail(c, LWACM_E_ARG, "dtype must be F32 or F64");
    if (where != LWACM_DEVICE && where != LWACM_HOST) return fail(c, LWACM_E_ARG, "bad location");
    const void *src[3] = {gx, gy, gz};
    const size_t sb = dtype == LWACM_F64 ? 8 : 4;
    const size_t nbytes = (size_t)c->N * sb;
    for (int a = 0; a < c->D; ++a) {
        char *dst = c->ws + c->off_ff + (size_t)a * c->Nal * 4;
        if (dtype == LWACM_F32) {
            CK(c, cudaMemcpyAsync(dst, src[a], nbytes,
                                  where == LWACM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  c->stream),
               "force field copy");
            continue;
        }
        const void *dsrc = src[a];
        if (where == LWACM_HOST) {
            CK(c, cudaMemcpyAsync(c->ws + c->off_stage, src[a], nbytes, cudaMemcpyHostToDevice, c->stream),
               "H2D stage");
            dsrc = c->ws + c->off_stage;
        }
        CK(c, launch_convert_in(STORE_F32, LWACM_F64, dsrc, dst, c->N, c->stream), "force field convert");
    }
    if (!c->ff_active) {
        c->ff_active = true;
        choose_kernel(c);
        drop_graphs(c);
    }
    return LWACM_OK;
}

lwacm_status lwacm_prepare(lwacm_ctx *c, long long n) {
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (n < 0) return fail(c, LWACM_E_ARG, "negative step count");
    if (c->sr && c->kernel != 5)
        return fail(c, LWACM_E_UNSUPPORTED, "stochastic rounding needs the half-row kernel (the plain periodic scheme)");
    const int chunk = c->graph_chunk;
    if (c->nbatch && c->batch_mode == 1) return LWACM_OK;  // one persistent launch, no graph
    if (chunk <= 0 || n < chunk) return LWACM_OK;
    const int par = c->cur;
    if (c->gexec[par] && c->gchunk[par] == chunk) return LWACM_OK;
    if (c->gexec[par]) {
        cudaGraphExecDestroy(c->gexec[par]);
        c->gexec[par] = nullptr;
    }
    return build_graph(c, par, chunk);
}

lwacm_status lwacm_step(lwacm_ctx *c, long long n) {
    const Range range("lwacm_step");
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (n < 0) return fail(c, LWACM_E_ARG, "negative step count");
    if (c->sr && c->kernel != 5)  // an option set later may have ruled the half-row kernel out
        return fail(c, LWACM_E_UNSUPPORTED, "stochastic rounding needs the half-row kernel (the plain periodic scheme)");
    if (c->nbatch && c->batch_mode == 1) {
        if (n == 0) return LWACM_OK;
        CK(c, launch_batch_persistent(c->Q, c->storage, bufp(c, 0), bufp(c, 1), batch_params(c), n, c->cur,
                                      c->stream),
           "persistent batch launch");
        c->cur ^= (int)(n & 1);
        c->steps += n;
        return LWACM_OK;
    }
    long long left = n;
    const int chunk = c->graph_chunk;
    if (chunk > 0 && left >= chunk) {
        // graphs are replayed on the bound stream; capture needs a private stream
        const int par = c->cur;
        if (!c->gexec[par] || c->gchunk[par] != chunk) {
            if (c->gexec[par]) {
                cudaGraphExecDestroy(c->gexec[par]);
                c->gexec[par] = nullptr;
            }
            s = build_graph(c, par, chunk);
            if (s != LWACM_OK) return s;
        }
        while (left >= chunk) {
            CK(c, cudaGraphLaunch(c->gexec[par], c->stream), "graph launch");
            left -= chunk;
            c->steps += chunk;  // chunk is even: parity unchanged
        }
    }
    for (; left > 0; --left) {
        CK(c, enqueue_step(c, c->cur, c->stream), "step launch");
        c->cur ^= 1;
        c->steps += 1;
    }
    return LWACM_OK;
}

lwacm_status lwacm_fields(lwacm_ctx *c, void **d, void **ux, void **uy, void **uz, int *dtype,
                          long long *pitch) {
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    char *b = (char *)bufp(c, c->cur);
    const size_t fb = field_bytes(c);
    if (d) *d = b;
    if (ux) *ux = b + fb;
    if (uy) *uy = b + 2 * fb;
    if (uz) *uz = c->Q == 19 ? b + 3 * fb : nullptr;
    if (dtype) *dtype = c->storage;
    if (pitch) *pitch = c->nx;
    return LWACM_OK;
}

static lwacm_status get_fields(lwacm_ctx *c, void *d, void *ux, void *uy, void *uz, int dtype, int where,
                               bool sync) {
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (!d || !ux || !uy || (c->Q == 19 && !uz))
        return fail(c, LWACM_E_ARG, "field pointers: d, ux, uy required; uz for D3Q19");
    if (dtype != LWACM_F32 && dtype != LWACM_F64) return fail(c, LWACM_E_ARG, "dtype must be F32 or F64");
    if (where != LWACM_DEVICE && where != LWACM_HOST) return fail(c, LWACM_E_ARG, "bad location");
    void *dst[4] = {d, ux, uy, uz};
    const size_t nbytes = (size_t)c->N * (dtype == LWACM_F64 ? 8 : 4);
    const char *b = (const char *)bufp(c, c->cur);
    for (int f = 0; f < c->nf; ++f) {
        const char *fs = b + (size_t)f * field_bytes(c);
        if (where == LWACM_HOST && dtype == LWACM_F32 && c->storage == LWACM_F32) {
            CK(c, cudaMemcpyAsync(dst[f], fs, nbytes, cudaMemcpyDeviceToHost, c->stream), "D2H");
            continue;
        }
        void *ddst = where == LWACM_HOST ? (void *)(c->ws + c->off_stage) : dst[f];
        CK(c, launch_convert_out(c->storage, dtype, fs, ddst, c->N, c->stream), "convert out");
        if (where == LWACM_HOST)
            CK(c, cudaMemcpyAsync(dst[f], ddst, nbytes, cudaMemcpyDeviceToHost, c->stream), "D2H stage");
    }
    if (where == LWACM_HOST && sync) CK(c, cudaStreamSynchronize(c->stream), "sync");
    return LWACM_OK;
}

lwacm_status lwacm_get_fields(lwacm_ctx *c, void *d, void *ux, void *uy, void *uz, int dtype,
                              int where) {
    const Range range("lwacm_get_fields");
    return get_fields(c, d, ux, uy, uz, dtype, where, true);
}

lwacm_status lwacm_get_fields_async(lwacm_ctx *c, void *d, void *ux, void *uy, void *uz, int dtype,
                                    int where) {
    const Range range("lwacm_get_fields_async");
    return get_fields(c, d, ux, uy, uz, dtype, where, false);
}

lwacm_status lwacm_set_scalar(lwacm_ctx *c, const void *T, int dtype, int where) {
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (c->alpha == 0) return fail(c, LWACM_E_STATE, "no scalar (LWACM_OPT_SCALAR_ALPHA before bind)");
    if (!T) return fail(c, LWACM_E_ARG, "null scalar");
    if (dtype != LWACM_F32 && dtype != LWACM_F64) return fail(c, LWACM_E_ARG, "dtype must be F32 or F64");
    if (where != LWACM_DEVICE && where != LWACM_HOST) return fail(c, LWACM_E_ARG, "bad location");
    char *fd = (char *)bufp(c, c->cur) + (size_t)c->nf * field_bytes(c);
    const size_t nbytes = (size_t)c->N * (dtype == LWACM_F64 ? 8 : 4);
    if (where == LWACM_HOST && dtype == LWACM_F32 && c->storage == LWACM_F32) {
        CK(c, cudaMemcpyAsync(fd, T, nbytes, cudaMemcpyHostToDevice, c->stream), "H2D");
        return LWACM_OK;
    }
    const void *src = T;
    if (where == LWACM_HOST) {
        CK(c, cudaMemcpyAsync(c->ws + c->off_stage, T, nbytes, cudaMemcpyHostToDevice, c->stream), "H2D stage");
        src = c->ws + c->off_stage;
    }
    CK(c, launch_convert_in(c->storage, dtype, src, fd, c->N, c->stream), "convert in");
    return LWACM_OK;
}

static lwacm_status get_extra(lwacm_ctx *c, void *T, int dtype, int where) {
    if (!T) return fail(c, LWACM_E_ARG, "null output");
    if (dtype != LWACM_F32 && dtype != LWACM_F64) return fail(c, LWACM_E_ARG, "dtype must be F32 or F64");
    if (where != LWACM_DEVICE && where != LWACM_HOST) return fail(c, LWACM_E_ARG, "bad location");
    const char *fs = (const char *)bufp(c, c->cur) + (size_t)c->nf * field_bytes(c);
    const size_t nbytes = (size_t)c->N * (dtype == LWACM_F64 ? 8 : 4);
    if (where == LWACM_HOST && dtype == LWACM_F32 && c->storage == LWACM_F32) {
        CK(c, cudaMemcpyAsync(T, fs, nbytes, cudaMemcpyDeviceToHost, c->stream), "D2H");
    } else {
        void *ddst = where == LWACM_HOST ? (void *)(c->ws + c->off_stage) : T;
        CK(c, launch_convert_out(c->storage, dtype, fs, ddst, c->N, c->stream), "convert out");
        if (where == LWACM_HOST)
            CK(c, cudaMemcpyAsync(T, ddst, nbytes, cudaMemcpyDeviceToHost, c->stream), "D2H stage");
    }
    if (where == LWACM_HOST) CK(c, cudaStreamSynchronize(c->stream), "sync");
    return LWACM_OK;
}

lwacm_status lwacm_get_scalar(lwacm_ctx *c, void *T, int dtype, int where) {
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (c->alpha == 0) return fail(c, LWACM_E_STATE, "no scalar (LWACM_OPT_SCALAR_ALPHA before bind)");
    return get_extra(c, T, dtype, where);
}

lwacm_status lwacm_get_trace(lwacm_ctx *c, void *T, int dtype, int where) {
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (!c->bulk) return fail(c, LWACM_E_STATE, "no bulk-viscosity variant (LWACM_OPT_BULK_GAMMA before bind)");
    return get_extra(c, T, dtype, where);
}

lwacm_status lwacm_diagnostics(lwacm_ctx *c, double out[8]) {
    const Range range("lwacm_diagnostics");
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (!out) return fail(c, LWACM_E_ARG, "null output");
    double *partial = (double *)(c->ws + c->off_partial);
    double *res = (double *)(c->ws + c->off_diag);
    CK(c, launch_diagnostics(c->storage, bufp(c, c->cur), c->Nal, c->N, c->Q == 19 ? 1 : 0,
                             partial, res, c->stream),
       "diagnostics");
    double h[kDiagValues];
    CK(c, cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "D2H diag");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
    for (int k = 0; k < 8; ++k) out[k] = h[k];
    out[5] = std::sqrt(h[5]);
    if (h[8] != 0.0) return fail(c, LWACM_E_NONFINITE, "non-finite values in the fields");
    return LWACM_OK;
}

lwacm_status lwacm_adjoint_workspace_bytes(const lwacm_ctx *c, long long T, int stride,
                                           size_t *bytes) {
    if (!c || !bytes || T < 0 || stride < 0) return LWACM_E_ARG;
    *bytes = adj_layout(c, T, stride).bytes;
    return LWACM_OK;
}

lwacm_status lwacm_forward_record(lwacm_ctx *c, long long T, int stride, void *ws, size_t bytes) {
    const Range range("lwacm_forward_record");
    lwacm_status s = ready(c, true);
    if (s != LWACM_OK) return s;
    if (T < 0 || stride < 0 || !ws) return fail(c, LWACM_E_ARG, "T >= 0, stride >= 0, workspace required");
    if (((uintptr_t)ws) % kAlign) return fail(c, LWACM_E_ARG, "adjoint workspace not 256-byte aligned");
    if (c->storage != LWACM_F32 || c->nbatch)
        return fail(c, LWACM_E_UNSUPPORTED, "the adjoint needs one domain with FP32 storage");
    if (c->ff_active) return fail(c, LWACM_E_UNSUPPORTED, "the adjoint does not take a force field");
    if (c->nu_p > 0 && c->nu_p != c->nu) return fail(c, LWACM_E_UNSUPPORTED, "the adjoint needs omega_p = omega");
    if (c->semi) return fail(c, LWACM_E_UNSUPPORTED, "the adjoint is for the explicit update");
    if (c->nsc) return fail(c, LWACM_E_UNSUPPORTED, "the adjoint does not carry the scalar");
    const AdjLayout L = adj_layout(c, T, stride);
    if (bytes < L.bytes) return fail(c, LWACM_E_NOMEM, "adjoint workspace smaller than lwacm_adjoint_workspace_bytes");
    c->adj = (char *)ws;
    c->adj_bytes = bytes;
    const size_t sb = (size_t)c->Nal * 4 * c->nf;
    c->rec_last_kept = false;
    for (long long k = 0; k < L.K; ++k) {
        char *ck = c->adj + L.ckpt + k * L.state;
        CK(c, cudaMemcpyAsync(ck, bufp(c, c->cur), sb, cudaMemcpyDeviceToDevice, c->stream), "checkpoint copy");
        const long long n = std::min<long long>(L.S, T - k * L.S);
        if (n > 0 && k == L.K - 1) {
            // the last segment steps through the segment buffer, whose states the
            // backward sweep then reads without recomputing them; its last state
            // becomes the context's current state
            char *seg = c->adj + L.seg;
            for (long long j = 0; j < n; ++j)
                CK(c, step_between(c, j == 0 ? ck : seg + j * L.state, seg + (j + 1) * L.state, c->stream),
                   "recorded step");
            CK(c, cudaMemcpyAsync(bufp(c, c->cur), seg + n * L.state, sb, cudaMemcpyDeviceToDevice, c->stream),
               "final state");
            c->steps += n;
            c->rec_last_kept = true;
        } else if (n > 0) {
            s = lwacm_step(c, n);
            if (s != LWACM_OK) return s;
        }
    }
    c->rec_T = T;
    c->rec_S = L.S;
    return LWACM_OK;
}

lwacm_status lwacm_backward(lwacm_ctx *c, const void *ld, const void *lux, const void *luy,
                            const void *luz, int dtype, void *gd, void *gux, void *guy, void *guz,
                            double *g_nu) {
    const Range range("lwacm_backward");
    lwacm_status s = ready(c, false);
    if (s != LWACM_OK) return s;
    if (c->rec_T < 0 || !c->adj) return fail(c, LWACM_E_STATE, "no recorded run (call lwacm_forward_record)");
    if (!ld || !lux || !luy || !gd || !gux || !guy || !g_nu || (c->Q == 19 && (!luz || !guz)))
        return fail(c, LWACM_E_ARG, "null argument");
    if (dtype != LWACM_F32 && dtype != LWACM_F64) return fail(c, LWACM_E_ARG, "dtype must be F32 or F64");
    const long long T = c->rec_T;
    const AdjLayout L = adj_layout(c, T, c->rec_S);
        const size_t fb = (size_t)c->Nal * 4;
    char *A = c->adj;
    // lambda in and out in lam0; (Dbar, Jbar) alternate between the other two
    float *lam0 = (float *)(A + L.lam);
    float *dj[2] = {(float *)(A + L.lam + L.state), (float *)(A + L.dj)};
    double *part = (double *)(A + L.part), *total = (double *)(A + L.total);
    unsigned *done = (unsigned *)(A + L.total + 8);
    const void *lin[4] = {ld, lux, luy, luz};
    for (int f = 0; f < c->nf; ++f)
        CK(c, launch_convert_in(STORE_F32, dtype, lin[f], (char *)lam0 + f * fb, c->N, c->stream), "lambda in");
    CK(c, cudaMemsetAsync(total, 0, 16, c->stream), "clear dnu");
    const StepParams p = params(c);
    int cur = 0;
    for (long long k = L.K - 1; k >= 0; --k) {
        const long long t0 = k * L.S;
        const long long len = std::min<long long>(L.S, T - t0);
        char *seg = A + L.seg;
        // the state at step j of the segment: the checkpoint itself for j = 0
        char *ck = A + L.ckpt + k * L.state;
        auto state = [&](long long j) { return j == 0 ? ck : seg + j * L.state; };
        if (!(k == L.K - 1 && c->rec_last_kept))
            for (long long j = 0; j < len; ++j)
                CK(c, step_between(c, state(j), seg + (j + 1) * L.state, c->stream), "segment recompute");
        for (long long j = len - 1; j >= 0; --j) {
            const bool first = k == L.K - 1 && j == len - 1, last = k == 0 && j == 0;
            CK(c, launch_adjoint_step(c->Q, (const float *)state(j), (const float *)state(j + 1),
                                      first ? lam0 : nullptr, dj[cur], last ? nullptr : dj[1 - cur], lam0, p, part,
                                      done, total, c->stream),
               "adjoint step");
            cur ^= 1;
        }
    }
    // a recomputed segment overwrote the kept one (a second backward recomputes it)
    c->rec_last_kept = c->rec_last_kept && L.K == 1;
    void *gout[4] = {gd, gux, guy, guz};
    for (int f = 0; f < c->nf; ++f) {
        if (dtype == LWACM_F32)
            CK(c, cudaMemcpyAsync(gout[f], (char *)lam0 + f * fb, (size_t)c->N * 4, cudaMemcpyDeviceToDevice,
                                  c->stream),
               "gradient out");
        else
            CK(c, launch_convert_out(STORE_F32, LWACM_F64, (char *)lam0 + f * fb, gout[f], c->N, c->stream),
               "gradient out");
    }
    double h = 0.0;
    CK(c, cudaMemcpyAsync(&h, total, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "dnu out");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
    *g_nu = h;
    return LWACM_OK;
}

lwacm_status lwacm_step_count(const lwacm_ctx *c, long long *steps) {
    if (!c || !steps) return LWACM_E_ARG;
    *steps = c->steps;
    return LWACM_OK;
}

lwacm_status lwacm_sync(lwacm_ctx *c) {
    lwacm_status s = ready(c, false);
    if (s != LWACM_OK) return s;
    int err = 0;
    CK(c, cudaMemcpyAsync(&err, c->ws + c->off_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "read error word");
    CK(c, cudaStreamSynchronize(c->stream), "sync");
    CK(c, cudaGetLastError(), "async error");
    if (err) return fail(c, LWACM_E_TIMEOUT, "a device-side wait gave up (data copy did not arrive)");
    return LWACM_OK;
}

lwacm_status lwacm_autotune(lwacm_ctx *c, const char *cache_path, int trial_steps, char *report,
                            size_t report_bytes) {
    const Range range("lwacm_autotune");
    lwacm_status s = ready(c, false);
    if (s != LWACM_OK) return s;
    if (c->has_fields)
        return fail(c, LWACM_E_STATE, "autotune runs on a fresh context: after lwacm_bind, before lwacm_set_fields");
    if (trial_steps < 0 || trial_steps > 100000) return fail(c, LWACM_E_ARG, "trial_steps must be in [0, 100000]");
    const long long T = trial_steps ? trial_steps : 256;
    const std::string key = tune_key(c);
    std::vector<Cand> cands = tune_candidates(c);
    std::vector<double> times(cands.size(), -1.0);
    std::vector<std::string> names(cands.size());
    TuneChoice best;
    std::string source = "measured";
    bool stored = false;
    TuneChoice hit;
    int best_i = -1;
    if (cache_path && tune_cache_lookup(cache_path, key, &hit)) {
        for (size_t i = 0; i < cands.size(); ++i)
            if (cands[i].kernel == hit.kernel && cands[i].tile == hit.tile && cands[i].mode == hit.mode)
                best_i = (int)i;
        if (best_i >= 0 && apply_cand(c, cands[best_i]) == LWACM_OK) {
            best = hit;
            source = "cache";
        } else {
            best_i = -1;
        }
    }
    if (best_i < 0) {
        // time every candidate from the rest state (d = 0, u = 0: a fixed point)
        const int keep_kernel = c->kernel_opt, keep_tile = c->batch_shape, keep_mode = c->batch_mode;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CK(c, cudaEventCreate(&e0), "event");
        CK(c, cudaEventCreate(&e1), "event");
        const long long warm = std::max(8, c->graph_chunk);
        lwacm_status st = LWACM_OK;
        for (size_t i = 0; i < cands.size() && st == LWACM_OK; ++i) {
            if (apply_cand(c, cands[i]) != LWACM_OK) continue;
            names[i] = c->kname;
            st = tune_zero_state(c);
            if (st == LWACM_OK) st = lwacm_step(c, warm);
            if (st == LWACM_OK) st = lwacm_sync(c);
            if (st != LWACM_OK) break;
            cudaEventRecord(e0, c->stream);
            st = lwacm_step(c, T);
            cudaEventRecord(e1, c->stream);
            if (st == LWACM_OK) st = lwacm_sync(c);
            float ms = 0.f;
            if (st == LWACM_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
                times[i] = 1e3 * ms / (double)T;
                if (best_i < 0 || times[i] < times[best_i]) best_i = (int)i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->has_fields = false;
        c->steps = 0;
        c->cur = 0;
        if (st != LWACM_OK) return st;
        if (best_i < 0) {
            c->kernel_opt = keep_kernel;
            c->batch_shape = keep_tile;
            c->batch_mode = keep_mode;
            choose_kernel(c);
            return fail(c, LWACM_E_UNSUPPORTED, "no candidate configuration ran");
        }
        best.kernel = cands[best_i].kernel;
        best.tile = cands[best_i].tile;
        best.mode = cands[best_i].mode;
        best.us = times[best_i];
        s = apply_cand(c, cands[best_i]);
        if (s != LWACM_OK) return s;
        if (cache_path) stored = tune_cache_store(cache_path, key, best);
    }
    if (report && report_bytes) {
        std::string r = "{\"key\": \"" + key + "\", \"source\": \"" + source + "\", \"choice\": {\"name\": \"" +
                        c->kname + "\", \"kernel\": " + std::to_string(best.kernel) +
                        ", \"tile\": " + std::to_string(best.tile) + ", \"mode\": " + std::to_string(best.mode) +
                        ", \"us_per_step\": " + std::to_string(best.us) + "}, \"cache_written\": " +
                        (stored ? "true" : "false") + ", \"candidates\": [";
        bool first = true;
        for (size_t i = 0; i < cands.size(); ++i) {
            if (times[i] < 0) continue;
            r += std::string(first ? "" : ", ") + "{\"name\": \"" + names[i] + "\", \"kernel\": " +
                 std::to_string(cands[i].kernel) + ", \"tile\": " + std::to_string(cands[i].tile) +
                 ", \"mode\": " + std::to_string(cands[i].mode) + ", \"us_per_step\": " + std::to_string(times[i]) +
                 "}";
            first = false;
        }
        r += "]}";
        std::snprintf(report, report_bytes, "%s", r.c_str());
    }
    return LWACM_OK;
}

const char *lwacm_last_error(const lwacm_ctx *c) { return c ? c->err.c_str() : "null context"; }

const char *lwacm_kernel_name(const lwacm_ctx *c) { return c ? c->kname.c_str() : ""; }

void lwacm_destroy(lwacm_ctx *c) {
    if (!c) return;
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

}  // extern "C"
