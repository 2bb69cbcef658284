// Host orchestration and the C ABI (include/dsbcg.h).
//
// A solve (Sec. 3) runs as:
//   1. pack B into the internal high-precision layout; ||b_i||;
//   2. joint inner solve: the block Lanczos process of A seeded with B, and
//      every shift's block root-free Cholesky recurrences, in the storage
//      precision (FP32 arithmetic for FP32/BF16/FP16 storage, FP64 for FP64);
//      each block step is a fixed sequence of kernels that read the block
//      widths and the convergence state from a device-resident control block,
//      so the host enqueues steps without synchronising and only polls the
//      `done` flag every `poll_every` steps;
//   3. true residuals r_ij = b_i - (sigma_j + A) x_ij (reliable update) in
//      high precision: FP64 for FP64 storage, double-float (pairs of FP32
//      words, 48-bit significands, FP32 pipes) for the reduced storages,
//      because GB300 runs FP64 arithmetic at 1/64 of the FP32 rate;
//   4. every shift with a residual above tol is restarted on its own true
//      residual (block CG on sigma_j I + A, same kernels with s = 1) and its
//      high-precision solution corrected, until every ||r_ij|| <= tol ||b_i||
//      or the restart cap is reached.
// The paper's own code runs in FP64 only (Sec. 4); the reduced-precision
// inner iteration with high-precision true-residual restarts is a
// GB300-specific addition.  Restarting is valid because the Galerkin iterate
// of a restarted process is again of the form of Eq. 3.2 for the new
// right-hand side.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <cstdlib>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/dsbcg.h"
#include "kernels.h"

// NVTX ranges (header-only NVTX 3; no-ops unless a profiler attaches)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define DSBCG_HAVE_NVTX 1
#endif

using namespace dsbcg;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct KEvent {
    int cls;
    cudaEvent_t a, b;
};

// One inner solve (one block Lanczos process with s_in shifts): its device
// buffers, control block and stream.  Lane 0 is the joint solve of all shifts
// on the context's stream; the per-shift restarts of the refinement loop run
// on lane 0 and on further one-shift lanes with their own streams, so that
// the m x m kernels of one restart (latency-bound) overlap the streaming
// kernels of the others.
struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t ready = nullptr;                  // own lanes: main-stream work they wait for
    void *vring = nullptr, *zw = nullptr, *y = nullptr, *P = nullptr, *Xin = nullptr;
    void* eotmp = nullptr;                        // Schur operator: even-parity half fields
    double2* rhs = nullptr;                       // gathered right-hand sides (high precision)
    double* partials = nullptr;
    int nblk = 0;
    dsbcg::SmallState* ss = nullptr;
    dsbcg::Ctl* ctl = nullptr;
    double2* G = nullptr;
    double* diag = nullptr;
    void *coef_a = nullptr, *coef_bh = nullptr, *coefS = nullptr, *coefU = nullptr, *coefL = nullptr;
    int *active = nullptr, *conv_step = nullptr;
    double *res = nullptr, *sigma = nullptr, *target = nullptr;
    dsbcg::Ctl* h_ctl = nullptr;                  // pinned
    int* h_conv = nullptr;                        // pinned
    int* h_active = nullptr;                      // pinned (joint lane): shifts updated in the last step
    // the inner solve in progress
    int m_in = 0, s_in = 0, prec = 0, step = 0, max_steps = 0, freeze = 0, poll_every = 1;
    // block steps per shift-update chunk (the basis ring holds chunk + 1
    // blocks; coefficient tiles and active flags chunk slots) and the last
    // step already folded into P and X
    int chunk = 1, k0 = 0;
    int chunk_used = 1;                           // the running inner solve's chunk (<= chunk)
    int sfp64 = 1;                                // m x m scalar: FP64 (1) or double-float (0)
    double dtol = 0;
    bool running = false;
};

}  // namespace

struct dsbcg_ctx {
    Geom g;
    size_t V = 0, n = 0, ld = 0;
    size_t Vf = 0;                       // sites of a field: V, or V / 2 for the Schur operator
    int schur = 0;                       // 1: the even-odd Schur operator on the odd sites
    double kappa = 0;
    cudaStream_t st = nullptr;
    double2* gauge64 = nullptr;          // canonical copy of the links (device)
    void* links[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // per Prec (PDD: double-float)
    // 12-real copies (rows 0, 1) for FP32 / 16-bit storage, packed when every
    // link of the field is in SU(3) to 1e-10 (su3); the stencil rebuilds row 2
    void* links12[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool su3 = false;
    float hscale = 1.f;
    bool gauge_ok = false;               // gauge64 holds a checked field and links[] were packed from it
    // refinement stream (true residuals, restarts' bookkeeping) beside the
    // context's stream, and the events that order the two; created on first use
    cudaStream_t rst = nullptr;
    cudaEvent_t ev_joint = nullptr, ev_ref = nullptr;
    // CTAs of an FP64 true-residual stencil launch (0: one per work item);
    // set on first use
    int resid_ctas = -1;
    // cap on the shift-update chunk (test hook; 0: automatic)
    int force_chunk = 0;
    int debug_first_wait = -1;           // test hook of the block Gram kernel (dsbcg_debug_first_wait)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<KEvent> ev_live;
    double kms[8] = {0};
    long long klaunch[8] = {0};
    double kbytes[8] = {0};
    double kflops[8] = {0};
    // workspace
    std::vector<void*> allocs;
    struct WS {
        int m = 0, s = 0, prec = -1;
        int nbb = 0;                     // right-hand-side blocks in B64 (1, or s for per-shift B)
        void *vring = nullptr, *zw = nullptr, *y = nullptr;       // storage precision
        void* eotmp = nullptr;                                    // Schur: even-parity half fields
        double2* T64c = nullptr;                                  // Schur: high-precision half fields
        void *P = nullptr, *Xin = nullptr;                        // work precision
        double2 *B64 = nullptr, *X64 = nullptr, *R64 = nullptr, *T64a = nullptr, *T64b = nullptr, *rhs = nullptr;
        double2 *Xg = nullptr, *Bg = nullptr;
        double* partials = nullptr;
        double* rpart = nullptr;
        SmallState* ss = nullptr;
        Ctl* ctl = nullptr;
        double2 *G = nullptr, *alpha = nullptr;
        double *diag = nullptr, *yy = nullptr;
        void *coef_a = nullptr, *coef_bh = nullptr, *coefS = nullptr, *coefU = nullptr, *coefL = nullptr;
        int *active = nullptr, *conv_step = nullptr;
        double *res = nullptr, *sigma = nullptr, *target = nullptr, *norms = nullptr;
        double* coefR = nullptr;         // rational-combination weights alpha_0..alpha_s
        int* flag = nullptr;
        Ctl* h_ctl = nullptr;            // pinned
        double* h_norms = nullptr;       // pinned
        int* h_conv = nullptr;           // pinned
        int* h_active = nullptr;         // pinned
        int nblk = 0, rblk = 0;
        std::vector<void*> mem;
        std::vector<Lane> lanes;        // [0]: the joint solve's buffers; then refinement lanes
        std::vector<void*> pinned;      // refinement lanes' pinned words
    } ws;
};

namespace {

// one named NVTX range for the lifetime of the object (host thread)
struct Range {
    explicit Range(const char* name) {
#ifdef DSBCG_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~Range() {
#ifdef DSBCG_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

#define CK(x)                                              \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) {                           \
            fprintf(stderr, "dsbcg: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? DSBCG_ERR_OOM : DSBCG_ERR_CUDA; \
        }                                                  \
    } while (0)

#define CKS(x)                                    \
    do {                                          \
        dsbcg_status s_ = (x);                    \
        if (s_ != DSBCG_OK) return s_;            \
    } while (0)

inline int work_prec(int p) { return p == P64 ? P64 : P32; }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device address of page-locked host memory mapped into the device address
// space (nullptr for device, pageable or unmapped memory)
void* mapped_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

dsbcg_status dmalloc(dsbcg_ctx* c, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        cudaGetLastError();
        fprintf(stderr, "dsbcg: device allocation of %zu bytes failed (%s; %zu of %zu bytes free)\n", bytes,
                cudaGetErrorString(e), fr, tot);
        return DSBCG_ERR_OOM;
    }
    c->ws.mem.push_back(*p);
    return DSBCG_OK;
}

void free_ws(dsbcg_ctx* c) {
    cudaStreamSynchronize(c->st);
    for (auto& L : c->ws.lanes) {
        if (L.st && L.st != c->st) {
            cudaStreamSynchronize(L.st);
            cudaStreamDestroy(L.st);
        }
        if (L.ready) cudaEventDestroy(L.ready);
    }
    for (void* p : c->ws.pinned) cudaFreeHost(p);
    for (void* p : c->ws.mem) cudaFree(p);
    c->ws.mem.clear();
    if (c->ws.h_ctl) cudaFreeHost(c->ws.h_ctl);
    if (c->ws.h_norms) cudaFreeHost(c->ws.h_norms);
    if (c->ws.h_conv) cudaFreeHost(c->ws.h_conv);
    if (c->ws.h_active) cudaFreeHost(c->ws.h_active);
    c->ws = dsbcg_ctx::WS();
}

size_t prec_elem_bytes(int p) { return (size_t)prec_bytes(p); }

dsbcg_status ensure_links(dsbcg_ctx* c, int prec) {
    if (c->links[prec]) return DSBCG_OK;
    void* p = nullptr;
    CK(cudaMalloc(&p, c->V * 36 * prec_elem_bytes(prec)));
    launch_pack_links(prec, p, c->gauge64, c->V, c->st);
    CK(cudaGetLastError());
    c->links[prec] = p;
    if (c->su3 && (prec == P32 || prec == PBF16 || prec == PF16) && !c->links12[prec]) {
        void* q = nullptr;
        CK(cudaMalloc(&q, c->V * 24 * prec_elem_bytes(prec)));
        launch_pack_links12(prec, q, c->gauge64, c->V, c->st);
        CK(cudaGetLastError());
        c->links12[prec] = q;
    }
    return DSBCG_OK;
}

// Block steps per shift-update chunk for a lane whose basis blocks take
// block_bytes: cmax (a power of two, at most CTL_HIST), halved while the
// ring of chunk + 1 blocks would take more than 1/frac of the device memory
// (at least 1: the per-step update with a two-block ring).
int chunk_steps(size_t block_bytes, int cmax, size_t frac) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int C = std::min(cmax, CTL_HIST);
    while (C > 1 && (size_t)(C + 1) * block_bytes > tot / frac) C /= 2;
    return C;
}

// Stream priorities: the refinement stream (true residuals, the start of
// every restart) takes the highest priority, the restart lanes the default.
// At 16^3 x 32 (m = s = 12) the solve took 333 ms this way, 337 ms with
// every stream at the default and 344 ms with the lanes at the highest.
int stream_prio(bool refinement) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return refinement ? greatest : least;
}

dsbcg_status ensure_ws(dsbcg_ctx* c, int m, int s, int prec, int nbb) {
    auto& w = c->ws;
    if (w.prec == prec && w.m == m && w.s >= s && w.nbb >= nbb) return DSBCG_OK;
    free_ws(c);
    const size_t ld = c->ld, n = c->n;
    const size_t fb = prec_elem_bytes(prec) * ld;           // storage field bytes
    const size_t wb = prec_elem_bytes(work_prec(prec)) * ld; // work field bytes
    const size_t db = sizeof(double2) * ld;
    (void)n;
    CKS(dmalloc(c, &w.zw, m * fb));
    CKS(dmalloc(c, &w.y, m * fb));
    if (c->schur) {
        CKS(dmalloc(c, &w.eotmp, m * fb));
        CKS(dmalloc(c, (void**)&w.T64c, m * db));
    }
    CKS(dmalloc(c, (void**)&w.P, (size_t)s * m * wb));
    CKS(dmalloc(c, (void**)&w.Xin, (size_t)s * m * wb));
    CKS(dmalloc(c, (void**)&w.B64, (size_t)nbb * m * db));
    CKS(dmalloc(c, (void**)&w.X64, (size_t)s * m * db));
    CKS(dmalloc(c, (void**)&w.R64, m * db));
    CKS(dmalloc(c, (void**)&w.T64a, m * db));
    CKS(dmalloc(c, (void**)&w.T64b, m * db));
    CKS(dmalloc(c, (void**)&w.rhs, m * db));
    CKS(dmalloc(c, (void**)&w.Xg, m * db));
    CKS(dmalloc(c, (void**)&w.Bg, m * db));
    w.nblk = gram_blocks(c->n, m);
    CKS(dmalloc(c, (void**)&w.partials, gram_partial_doubles(M_MAX) * sizeof(double)));
    w.rblk = residual_blocks(c->n);
    CKS(dmalloc(c, (void**)&w.rpart, (size_t)w.rblk * m * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.ss, small_state_bytes(s)));
    CKS(dmalloc(c, (void**)&w.ctl, sizeof(Ctl)));
    CKS(dmalloc(c, (void**)&w.G, M_MAX * M_MAX * sizeof(double2)));
    CKS(dmalloc(c, (void**)&w.alpha, M_MAX * M_MAX * sizeof(double2)));
    CKS(dmalloc(c, (void**)&w.diag, M_MAX * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.yy, M_MAX * sizeof(double)));
    const size_t tb = M_MAX * M_MAX * sizeof(double2);
    CKS(dmalloc(c, &w.coef_a, tb));
    CKS(dmalloc(c, &w.coef_bh, tb));
    CKS(dmalloc(c, &w.coefS, tb));

    CKS(dmalloc(c, (void**)&w.conv_step, (size_t)s * m * sizeof(int)));
    CKS(dmalloc(c, (void**)&w.res, (size_t)s * m * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.sigma, s * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.target, (size_t)s * m * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.norms, (size_t)(s + 1) * m * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.coefR, (size_t)(s + 1) * sizeof(double)));
    CKS(dmalloc(c, (void**)&w.flag, sizeof(int)));
    CK(cudaMallocHost((void**)&w.h_ctl, sizeof(Ctl)));
    CK(cudaMallocHost((void**)&w.h_norms, (size_t)(s + 1) * m * sizeof(double)));
    CK(cudaMallocHost((void**)&w.h_conv, (size_t)s * m * sizeof(int)));
    CK(cudaMallocHost((void**)&w.h_active, (size_t)s * sizeof(int)));
    // the basis ring and the per-step coefficient tiles and flags of the
    // shift-update chunks, last: a chunk that does not fit is halved, down
    // to the per-step update with a two-block ring
    int chunk0 = chunk_steps((size_t)m * fb, 16, 16);
    for (;; chunk0 /= 2) {
        void *ring = nullptr, *cu = nullptr, *cl = nullptr, *act = nullptr;
        if (cudaMalloc(&ring, (size_t)(chunk0 + 1) * m * fb) == cudaSuccess &&
            cudaMalloc(&cu, (size_t)chunk0 * s * tb) == cudaSuccess &&
            cudaMalloc(&cl, (size_t)chunk0 * s * tb) == cudaSuccess &&
            cudaMalloc(&act, (size_t)chunk0 * s * sizeof(int)) == cudaSuccess) {
            w.vring = ring;
            w.coefU = cu;
            w.coefL = cl;
            w.active = (int*)act;
            for (void* q : {ring, cu, cl, act}) w.mem.push_back(q);
            break;
        }
        cudaGetLastError();
        for (void* q : {ring, cu, cl, act})
            if (q) cudaFree(q);
        if (chunk0 == 1) {
            fprintf(stderr, "dsbcg: device allocation of the two-block basis ring (%zu bytes) failed\n",
                    (size_t)2 * m * fb);
            return DSBCG_ERR_OOM;
        }
    }
    w.m = m;
    w.s = s;
    w.prec = prec;
    w.nbb = nbb;
    Lane L0;
    L0.st = c->st;
    L0.vring = w.vring;
    L0.zw = w.zw;
    L0.y = w.y;
    L0.eotmp = w.eotmp;
    L0.P = w.P;
    L0.Xin = w.Xin;
    L0.rhs = w.rhs;
    L0.partials = w.partials;
    L0.nblk = w.nblk;
    L0.ss = w.ss;
    L0.ctl = w.ctl;
    L0.G = w.G;
    L0.diag = w.diag;
    L0.coef_a = w.coef_a;
    L0.coef_bh = w.coef_bh;
    L0.coefS = w.coefS;
    L0.coefU = w.coefU;
    L0.coefL = w.coefL;
    L0.active = w.active;
    L0.conv_step = w.conv_step;
    L0.res = w.res;
    L0.sigma = w.sigma;
    L0.target = w.target;
    L0.h_ctl = w.h_ctl;
    L0.h_conv = w.h_conv;
    L0.h_active = w.h_active;
    L0.chunk = chunk0;
    w.lanes.assign(1, L0);
    return DSBCG_OK;
}

// Add one-shift refinement lanes until there are `want` lanes (lane 0
// included) or device memory runs out; returns the number available.
int ensure_refine_lanes(dsbcg_ctx* c, int want) {
    auto& w = c->ws;
    const int m = w.m, prec = w.prec;
    const size_t fb = prec_elem_bytes(prec) * c->ld, wb = prec_elem_bytes(work_prec(prec)) * c->ld;
    const size_t db = sizeof(double2) * c->ld, tb = M_MAX * M_MAX * sizeof(double2);
    // a lane's buffers; lanes stop while a tenth of the device (at least
    // 4 GiB) would still be free, so that large lattices keep memory for the
    // caller
    const int chunk = chunk_steps((size_t)m * fb, 16, 64);
    const size_t lane_bytes = (c->schur ? 3 : 2) * m * fb + (size_t)(chunk + 1) * m * fb + 2 * m * wb + m * db +
                              gram_partial_doubles(M_MAX) * sizeof(double) + small_state_bytes(1) +
                              (4 + 2 * (size_t)chunk) * tb;
    while ((int)w.lanes.size() < want) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        const size_t reserve = std::max(tot / 10, (size_t)4 << 30);
        if (fr < lane_bytes + reserve) break;
        Lane L;
        L.chunk = chunk;
        bool ok = dmalloc(c, &L.vring, (size_t)(chunk + 1) * m * fb) == DSBCG_OK && dmalloc(c, &L.zw, m * fb) == DSBCG_OK &&
                  (!c->schur || dmalloc(c, &L.eotmp, m * fb) == DSBCG_OK) &&
                  dmalloc(c, &L.y, m * fb) == DSBCG_OK && dmalloc(c, &L.P, m * wb) == DSBCG_OK &&
                  dmalloc(c, &L.Xin, m * wb) == DSBCG_OK && dmalloc(c, (void**)&L.rhs, m * db) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.partials, gram_partial_doubles(M_MAX) * sizeof(double)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.ss, small_state_bytes(1)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.ctl, sizeof(Ctl)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.G, M_MAX * M_MAX * sizeof(double2)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.diag, M_MAX * sizeof(double)) == DSBCG_OK &&
                  dmalloc(c, &L.coef_a, tb) == DSBCG_OK && dmalloc(c, &L.coef_bh, tb) == DSBCG_OK &&
                  dmalloc(c, &L.coefS, tb) == DSBCG_OK && dmalloc(c, &L.coefU, (size_t)chunk * tb) == DSBCG_OK &&
                  dmalloc(c, &L.coefL, (size_t)chunk * tb) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.active, (size_t)chunk * sizeof(int)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.conv_step, m * sizeof(int)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.res, m * sizeof(double)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.sigma, sizeof(double)) == DSBCG_OK &&
                  dmalloc(c, (void**)&L.target, m * sizeof(double)) == DSBCG_OK;
        if (ok && cudaMallocHost((void**)&L.h_ctl, sizeof(Ctl)) == cudaSuccess) w.pinned.push_back(L.h_ctl);
        else ok = false;
        if (ok && cudaMallocHost((void**)&L.h_conv, m * sizeof(int)) == cudaSuccess) w.pinned.push_back(L.h_conv);
        else ok = false;
        if (ok && cudaStreamCreateWithPriority(&L.st, cudaStreamNonBlocking, stream_prio(false)) != cudaSuccess) {
            L.st = nullptr;
            ok = false;
        }
        if (ok && cudaEventCreateWithFlags(&L.ready, cudaEventDisableTiming) != cudaSuccess) {
            L.ready = nullptr;
            ok = false;
        }
        if (!ok) {
            // out of memory (or streams): run with the lanes there are; what
            // this attempt allocated stays in the workspace until it is freed
            cudaGetLastError();
            if (L.st) w.lanes.push_back(L);    // keeps the stream for free_ws; marked unusable below
            break;
        }
        L.nblk = gram_blocks(c->n, m);
        w.lanes.push_back(L);
    }
    int usable = 0;
    for (auto& L : w.lanes) {
        if (L.ready == nullptr && &L != &w.lanes[0]) break;
        ++usable;
    }
    return std::min(usable, std::max(1, want));
}

// ---- profiling -------------------------------------------------------------
cudaEvent_t ev_get(dsbcg_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
struct Prof {
    dsbcg_ctx* c;
    int cls;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Prof(dsbcg_ctx* c_, int cls_, int nlaunch = 1, cudaStream_t st_ = nullptr)
        : c(c_), cls(cls_), st(st_ ? st_ : c_->st) {
        if (c->profiling) {
            a = ev_get(c);
            cudaEventRecord(a, st);
        }
        c->klaunch[cls] += nlaunch;
    }
    ~Prof() {
        if (c->profiling) {
            cudaEvent_t b = ev_get(c);
            cudaEventRecord(b, st);
            c->ev_live.push_back({cls, a, b});
        }
    }
};
// Add the durations of completed launch-event pairs to their classes; pairs
// whose stream has not reached them yet stay for a later call.
void prof_collect(dsbcg_ctx* c) {
    std::vector<KEvent> pending;
    for (auto& k : c->ev_live) {
        float ms = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&ms, k.a, k.b);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            pending.push_back(k);
            continue;
        }
        if (e == cudaSuccess) c->kms[k.cls] += ms;
        else cudaGetLastError();
        c->ev_pool.push_back(k.a);
        c->ev_pool.push_back(k.b);
    }
    c->ev_live.swap(pending);
}

// ---- high-precision operator and true residual ------------------------------
// The true-residual loop runs on "high-precision" fields hp: FP64 (P64) for
// FP64 storage, double-float (PDD) for the reduced storages.  Both take 16
// bytes per complex, so buffers and byte offsets are the same; a PDD field
// is an FP32 hi plane and an FP32 lo plane of ld complex each.
inline size_t hp_ld(const dsbcg_ctx* c, int hp) { return hp == PDD ? 2 * c->ld : c->ld; }

// canonical complex128 fields <-> internal fields of any precision
void pack_any(dsbcg_ctx* c, int p, void* dst, const double2* src, int m) {
    if (p == PDD)
        launch_pack_pairs((float2*)dst, c->ld, src, m, c->Vf, c->st);
    else
        launch_pack_fields(p, dst, c->ld, src, m, c->Vf, c->hscale, c->st);
}
void unpack_any(dsbcg_ctx* c, int p, double2* dst, const void* src, int m, cudaStream_t st = nullptr) {
    if (!st) st = c->st;
    if (p == PDD)
        launch_unpack_pairs(dst, (const float2*)src, c->ld, m, c->Vf, st);
    else
        launch_unpack_fields(p, dst, src, c->ld, m, c->Vf, c->hscale, st);
}

// out = Dhat in (dag = 0) or Dhat^H in (dag = 1) on odd-parity half fields,
// Dhat = 1 - kappa^2 H_oe H_eo, Dhat^H = gamma_5 Dhat gamma_5; tmp receives
// the even-parity H_eo (gamma_5) in.  Two half-lattice passes.
void apply_dhat(dsbcg_ctx* c, int p, void* out, const void* in, void* tmp, size_t ld, int dag, const Ctl* ctl,
                int nf_static, int nf_max, float hs, cudaStream_t st, int cls) {
    {
        Prof q(c, cls, 1, st);
        launch_dslash_half(p, tmp, in, nullptr, ld, c->links[p], c->g, 0.0, 1.0, 0, dag, 0, ctl, nf_static, nf_max,
                           hs, st);
    }
    {
        Prof q(c, cls, 1, st);
        launch_dslash_half(p, out, tmp, in, ld, c->links[p], c->g, 1.0, -c->kappa * c->kappa, 1, 0, dag, ctl,
                           nf_static, nf_max, hs, st);
    }
}

// CTAs of the FP64 true-residual stencil.  The stencil is bound by the FP64
// pipe (2 FMA per clock per SM on GB300) and the latency of its neighbour
// loads; eight one-warp CTAs per SM keep it at full speed, so a grid of 8
// CTAs per SM striding over the work leaves the rest of each SM to the FP32
// kernels of the solve's other streams (DSBCG_RESIDUAL_CTAS_PER_SM overrides
// the 8; 0 lifts the cap).  At 16^3 x 32 with 12 fields the residual stencils
// of one solve take 130 ms at 8, 134 at 4 and 253 at 2 CTAs per SM (127
// uncapped), and the solve 353 ms at 8 against 364 uncapped.
int residual_ctas(dsbcg_ctx* c) {
    if (c->resid_ctas < 0) {
        int per_sm = 8, dev = 0, sms = 0;
        if (const char* e = getenv("DSBCG_RESIDUAL_CTAS_PER_SM")) per_sm = std::max(0, atoi(e));
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 0;
        }
        c->resid_ctas = per_sm * sms;
    }
    return c->resid_ctas;
}

// out = Op in for the fields of a block in precision p: the normal operator
// A = D^H D (two stencils; mid receives D in) or, on a context with the Schur
// operator, Ahat = Dhat^H Dhat (four half-lattice passes; mid receives
// Dhat in, tmp is scratch for even-parity half fields)
void apply_op(dsbcg_ctx* c, int p, void* out, void* mid, const void* in, void* tmp, size_t ld, const Ctl* ctl,
              int nf_static, int nf_max, float hs, cudaStream_t st, int cls) {
    if (c->schur) {
        apply_dhat(c, p, mid, in, tmp, ld, 0, ctl, nf_static, nf_max, hs, st, cls);
        apply_dhat(c, p, out, mid, tmp, ld, 1, ctl, nf_static, nf_max, hs, st, cls);
        return;
    }
    const int cap = (cls == DSBCG_KCLASS_RESIDUAL && p == P64) ? residual_ctas(c) : 0;
    {
        Prof q(c, cls, 1, st);
        launch_dslash(p, mid, in, ld, c->links[p], c->g, c->kappa, 0, ctl, nf_static, nf_max, hs, st, c->links12[p],
                      cap);
    }
    {
        Prof q(c, cls, 1, st);
        launch_dslash(p, out, mid, ld, c->links[p], c->g, c->kappa, 1, ctl, nf_static, nf_max, hs, st, c->links12[p],
                      cap);
    }
}

// link passes of one operator application: 2 (A) or 4 (Ahat); each pass
// reads every link once
inline double link_passes(const dsbcg_ctx* c) { return c->schur ? 4.0 : 2.0; }

// out = A in (or Ahat in) for nf high-precision fields (tmp receives D in), on stream st
void apply_Ahp(dsbcg_ctx* c, int hp, void* out, const void* in, void* tmp, int nf, cudaStream_t st) {
    apply_op(c, hp, out, tmp, in, c->ws.T64c, hp_ld(c, hp), nullptr, nf, nf, 1.f, st, DSBCG_KCLASS_RESIDUAL);
}

// r = b - sigma x - A x for m high-precision fields on stream st; squared
// column norms into h_out (host).  While the stream works, `idle` (if given)
// is called repeatedly (the solve keeps its lanes supplied meanwhile).
dsbcg_status true_residual(dsbcg_ctx* c, int hp, double2* r, const double2* b, const double2* x, int m,
                           double sigma, double* h_out, const std::function<dsbcg_status()>* idle, cudaStream_t st) {
    Range r_res("true residual");
    auto& w = c->ws;
    apply_Ahp(c, hp, w.T64b, x, w.T64a, m, st);
    {
        Prof p(c, DSBCG_KCLASS_RESIDUAL, 2, st);
        if (hp == PDD)
            launch_residual_pairs((float2*)r, (const float2*)b, (const float2*)x, (const float2*)w.T64b, c->ld, m,
                                  c->n, sigma, w.rpart, w.rblk, st);
        else
            launch_residual(r, b, x, w.T64b, c->ld, m, c->n, sigma, w.rpart, w.rblk, st);
        launch_reduce_cols(w.rpart, w.rblk, m, w.norms, st);
    }
    // two stencils (m fields in and out, links once each) + b, x, Ax in, r out
    c->kbytes[DSBCG_KCLASS_RESIDUAL] +=
        ((c->schur ? 14.0 : 8.0) * m * c->n + link_passes(c) * 36 * c->V) * sizeof(double2);
    CK(cudaMemcpyAsync(w.h_norms, w.norms, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (idle) {
        for (;;) {
            const cudaError_t e = cudaStreamQuery(st);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) CK(e);
            cudaGetLastError();
            CKS((*idle)());
        }
    }
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < m; ++i) h_out[i] = w.h_norms[i];
    return DSBCG_OK;
}

struct InnerResult {
    int steps = 0;
    long long mvms = 0;
    int deflations = 0;
    int final_rank = 0;
    int status = 0;
    bool converged = false;
};

// Inner solve on the right-hand sides `rhs` (m_in fields of precision
// rhs_prec, field stride rhs_ld, internal layout: FP64 for FP64 storage, the
// FP32 hi planes of double-float fields otherwise): for the shifts
// sig[0..s_in), L.Xin[j] (work precision) receives the iterate, targets are
// absolute residual norms per (j, i).  lane_start enqueues the
// initialisation; lane_enqueue the next poll_every block steps and a copy of
// the control block; lane_poll waits for them; lane_finish collects the
// result.  All work of a lane runs on its stream.
dsbcg_status lane_start(dsbcg_ctx* c, Lane& L, const void* rhs, int rhs_prec, size_t rhs_ld, int m_in,
                        const double* sig, int s_in, const double* targets, int prec, double dtol, int max_steps,
                        int freeze, int poll_every, int sfp64) {
    const int wp = work_prec(prec);
    const size_t ld = c->ld, n = c->n;
    const size_t fb = prec_elem_bytes(prec) * ld;
    const size_t wb = prec_elem_bytes(wp) * ld;
    cudaStream_t st = L.st;
    CK(cudaMemcpyAsync(L.sigma, sig, s_in * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(L.target, targets, (size_t)s_in * m_in * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(L.conv_step, 0xff, (size_t)s_in * m_in * sizeof(int), st));
    CK(cudaMemsetAsync(L.Xin, 0, (size_t)s_in * m_in * wb, st));
    // a0: G0 = B^H B (in the right-hand sides' precision), pivoted Cholesky
    // with deflation, V_1 = B S0.  A reduced-storage inner solve takes its
    // Gram and basis from an FP32 copy of FP64 right-hand sides, like every
    // other Gram of the solve (storage-precision fields, FP64 reduction and
    // m x m work): an FP64 Gram would be bound by the FP64 pipe (1/64 rate).
    // The lane's P block (work precision FP32, first written by step 1's
    // shift update, which starts from V_1) holds the copy.
    const void* grhs = rhs;
    int gprec = rhs_prec;
    size_t gld = rhs_ld;
    if (rhs_prec == P64 && prec != P64) {
        Prof p(c, DSBCG_KCLASS_OTHER, 1, st);
        launch_convert_64_32((float2*)L.P, ld, (const double2*)rhs, rhs_ld, m_in, n, st);
        c->kbytes[DSBCG_KCLASS_OTHER] += (double)m_in * n * (16.0 + 8.0);
        grhs = L.P;
        gprec = P32;
        gld = ld;
    }
    {
        Prof p(c, DSBCG_KCLASS_GRAM, 1, st);
        launch_gram(gprec, grhs, grhs, gld, n, nullptr, m_in, m_in, 1, 1, L.partials, L.nblk, 1.f, st);
    }
    {
        Prof p(c, DSBCG_KCLASS_SMALL, 2, st);
        launch_gram_reduce(L.partials, L.nblk, m_in, 1, 1, L.G, L.diag, nullptr, m_in, gprec != P64, st);
        launch_small_init(L.ss, L.ctl, L.G, L.diag, m_in, s_in, dtol, sfp64, st);
    }
    char* ring = (char*)L.vring;
    {
        Prof p(c, DSBCG_KCLASS_OTHER, 1, st);
        launch_init_basis(prec, ring + 1 * (size_t)m_in * fb, ld, grhs, gprec, gld, n, small_state_S(L.ss),
                          !sfp64, L.ctl, m_in, c->hscale, st);
    }
    c->kbytes[DSBCG_KCLASS_GRAM] += (double)m_in * n * prec_elem_bytes(gprec);
    c->kbytes[DSBCG_KCLASS_OTHER] += (double)m_in * n * (prec_elem_bytes(gprec) + prec_elem_bytes(prec));
    CK(cudaGetLastError());
    L.m_in = m_in;
    L.s_in = s_in;
    L.prec = prec;
    L.step = 0;
    L.k0 = 0;
    L.chunk_used = c->force_chunk > 0 ? std::min(L.chunk, c->force_chunk) : L.chunk;
    L.max_steps = max_steps;
    L.freeze = freeze;
    L.poll_every = poll_every;
    L.sfp64 = sfp64;
    L.dtol = dtol;
    L.running = true;
    return DSBCG_OK;
}

dsbcg_status lane_enqueue(dsbcg_ctx* c, Lane& L) {
    const int prec = L.prec, wp = work_prec(prec), m_in = L.m_in, s_in = L.s_in;
    const size_t ld = c->ld, n = c->n;
    const size_t fb = prec_elem_bytes(prec) * ld;
    const size_t cb = (wp == P64 ? 16 : 8) * (size_t)M_MAX * M_MAX;    // one coefficient tile
    cudaStream_t st = L.st;
    char* ring = (char*)L.vring;
    const int C = L.chunk_used, R = C + 1;
    auto slot = [&](int k) { return ring + (size_t)(k % R) * m_in * fb; };     // V_k
    // P_j and X_j take the steps L.k0 + 1 .. L.step (the chunk's executed ones)
    auto flush = [&]() {
        if (L.step == L.k0) return;
        Prof p(c, DSBCG_KCLASS_SHIFT, 1, st);
        launch_shift_chunk(prec, ring, (size_t)m_in * ld, R, ld, L.P, L.Xin, ld, n, s_in, m_in, L.ctl, m_in, L.k0,
                           C, L.coefU, L.coefL, L.active, c->hscale, st);
        L.k0 = L.step;
    };
    for (int q = 0; q < L.poll_every && L.step < L.max_steps; ++q) {
        const int step = ++L.step;
        void* Vk = slot(step);
        void* Vo = slot(step - 1);     // V_{k-1} (unused at k = 1)
        const int hs = (step - 1) % C;                 // this step's coefficient and flag slot
        apply_op(c, prec, L.y, L.zw, Vk, L.eotmp, ld, L.ctl, 0, m_in, c->hscale, st, DSBCG_KCLASS_DSLASH);
        {
            Prof p(c, DSBCG_KCLASS_GRAM, 1, st);
            // alpha_k = V_k^H A V_k is hermitian: the upper 4 x 4 tiles of
            // V_k^H Y only (their conjugates fill the lower ones)
            launch_gram(prec, Vk, L.y, ld, n, L.ctl, 0, m_in, 1, 1, L.partials, L.nblk, c->hscale, st,
                        c->debug_first_wait);
        }
        {
            Prof p(c, DSBCG_KCLASS_SMALL, 1, st);
            launch_small_alpha(L.ss, L.ctl, L.partials, L.nblk, m_in, wp, L.sfp64, L.coef_a, L.coef_bh, st);
        }
        if (update_gram_fits(prec, m_in)) {
            // W and its Gram W^H W in one pass over the rows
            Prof p(c, DSBCG_KCLASS_UPDATE, 1, st);
            launch_update_gram(prec, L.zw, L.y, Vk, Vo, ld, n, L.ctl, m_in, L.coef_a, L.coef_bh, L.partials, L.nblk,
                               c->hscale, st);
        } else {
            {
                Prof p(c, DSBCG_KCLASS_UPDATE, 1, st);
                launch_block_update(prec, L.zw, L.y, Vk, Vo, ld, n, L.ctl, m_in, L.coef_a, L.coef_bh, c->hscale,
                                    st);
            }
            {
                Prof p(c, DSBCG_KCLASS_GRAM, 1, st);
                launch_gram(prec, L.zw, L.zw, ld, n, L.ctl, 0, m_in, 1, 0, L.partials, L.nblk, c->hscale, st);
            }
        }
        {
            Prof p(c, DSBCG_KCLASS_SMALL, 1, st);
            launch_small_step(L.ss, L.ctl, L.partials, L.nblk, s_in, m_in, L.dtol, L.sigma, L.target, L.freeze, wp,
                              L.sfp64, L.coefS, (char*)L.coefU + (size_t)hs * s_in * cb,
                              (char*)L.coefL + (size_t)hs * s_in * cb, L.active + (size_t)hs * s_in, L.conv_step,
                              L.res, st);
        }
        {
            Prof p(c, DSBCG_KCLASS_UPDATE, 1, st);
            launch_v_update(prec, slot(step + 1), L.zw, ld, n, L.ctl, m_in, L.coefS, c->hscale, st);
        }
        {
            Prof p(c, DSBCG_KCLASS_SMALL, 1, st);
            launch_small_finish(L.ss, L.ctl, s_in, m_in, L.active + (size_t)hs * s_in, st);
        }
        if (L.step - L.k0 == C) flush();
    }
    flush();                           // P_j, X_j current at the end of every batch
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(L.h_ctl, L.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    if (L.h_active && L.step > 0)
        CK(cudaMemcpyAsync(L.h_active, L.active + (size_t)((L.step - 1) % C) * s_in, (size_t)s_in * sizeof(int),
                           cudaMemcpyDeviceToHost, st));
    return DSBCG_OK;
}

dsbcg_status lane_poll(dsbcg_ctx* c, Lane& L) {
    (void)c;
    CK(cudaStreamSynchronize(L.st));
    if (L.h_ctl->done || L.h_ctl->status != 0 || L.step >= L.max_steps) L.running = false;
    return DSBCG_OK;
}

// Run the started lanes to completion, enqueueing poll_every steps on each in
// turn before waiting on any, so that their kernels overlap on the GPU.
dsbcg_status run_lanes(dsbcg_ctx* c, Lane* const* lanes, int nl) {
    for (;;) {
        bool any = false;
        for (int i = 0; i < nl; ++i)
            if (lanes[i]->running) {
                CKS(lane_enqueue(c, *lanes[i]));
                any = true;
            }
        if (!any) break;
        for (int i = 0; i < nl; ++i)
            if (lanes[i]->running) CKS(lane_poll(c, *lanes[i]));
        prof_collect(c);
    }
    return DSBCG_OK;
}

dsbcg_status lane_finish(dsbcg_ctx* c, Lane& L, InnerResult* out, int step_offset, int* conv_step_host) {
    const int s_in = L.s_in, m_in = L.m_in, prec = L.prec, wp = work_prec(prec);
    const size_t n = c->n;
    CK(cudaMemcpyAsync(L.h_conv, L.conv_step, (size_t)s_in * m_in * sizeof(int), cudaMemcpyDeviceToHost, L.st));
    CK(cudaStreamSynchronize(L.st));
    if (conv_step_host) {
        for (int t = 0; t < s_in * m_in; ++t)
            conv_step_host[t] = L.h_conv[t] >= 0 ? L.h_conv[t] + step_offset : -1;
    }
    const Ctl& h = *L.h_ctl;
    {
        const double eb = (double)prec_elem_bytes(prec) * n, wbn = (double)prec_elem_bytes(wp) * n;
        // link entries read per stencil pass: 24 V with 12-real links (the
        // normal operator's FP32 / 16-bit stencil), else 36 V
        const double links = ((c->links12[prec] && !c->schur) ? 24.0 : 36.0) * c->V * (double)prec_elem_bytes(prec);
        // the Schur operator's four passes move 10 half fields per block
        // column (the counter counts the normal operator's 4)
        c->kbytes[DSBCG_KCLASS_DSLASH] += h.f_dslash * eb * (c->schur ? 2.5 : 1.0) + link_passes(c) * h.last_step * links;
        // f_gram counts V_k and Y for alpha and W for W^H W (3 m_k per step);
        // the fused update reads W once, for both
        c->kbytes[DSBCG_KCLASS_GRAM] += h.f_gram * eb * (update_gram_fits(prec, m_in) ? 2.0 / 3.0 : 1.0);
        c->kbytes[DSBCG_KCLASS_UPDATE] += h.f_update * eb;
        c->kbytes[DSBCG_KCLASS_SHIFT] += h.f_shift_s * eb + h.f_shift_w * wbn;
        c->kflops[DSBCG_KCLASS_SHIFT] += 8.0 * (double)h.f_shift_cmac * n;
    }
    out->steps = h.last_step;
    out->mvms = h.mvms;
    out->deflations = h.deflations;
    out->final_rank = h.mk;
    out->status = h.status;
    out->converged = h.done && h.status == 0;
    return DSBCG_OK;
}

double default_dtol(int prec) {
    switch (prec) {
        case P64: return 1e-7;
        case P32: return 1e-3;
        case PF16: return 1e-2;
        default: return 3e-2;
    }
}

}  // namespace

// ============================================================================
namespace {

// The solve behind dsbcg_solve, dsbcg_solve_rational and the adjoint solves of
// dsbcg_backward.  nbb = 1: one block B [m][n] for every shift (the joint
// block solve of Sec. 3 first); nbb = s: B is [s][m][n], shift j's own
// right-hand sides (each shift solved on a refinement lane, no joint solve).
// X (caller's [s][m][n]) may be NULL when rat is set; rat writes
// Y = alpha_0 B + sum_j alpha_j X_j (single-block B only).
struct RationalOut {
    double alpha0;
    const double* alpha;     // host [s]
    void* Y;                 // device or host complex128 [m][n]
};

dsbcg_status solve_core(dsbcg_ctx* c, int m, const void* B, int nbb, int s, const double* sigma, double tol,
                        const dsbcg_params* params, void* X, dsbcg_stats* stats, const RationalOut* rat) {
    Range r_solve("dsbcg_solve");
    auto t0 = std::chrono::steady_clock::now();
    if (!c || !B || !sigma || m < 1 || m > M_MAX || s < 1 || s > S_MAX) return DSBCG_ERR_ARG;
    if (!X && !rat) return DSBCG_ERR_ARG;
    if (nbb != 1 && (nbb != s || rat)) return DSBCG_ERR_ARG;
    if (rat) {
        if (!rat->Y || !rat->alpha || !isfinite(rat->alpha0)) return DSBCG_ERR_ARG;
        for (int j = 0; j < s; ++j)
            if (!isfinite(rat->alpha[j])) return DSBCG_ERR_ARG;
    }
    if (!c->gauge_ok) return DSBCG_ERR_ARG;
    if (!(tol >= 0.0) || !isfinite(tol)) return DSBCG_ERR_ARG;
    for (int j = 0; j < s; ++j)
        if (!(sigma[j] >= 0.0) || !isfinite(sigma[j])) return DSBCG_ERR_ARG;
    dsbcg_params prm;
    if (params) prm = *params;
    else dsbcg_params_default(&prm);
    const int prec = prm.storage;
    if (prec < 0 || prec > 3) return DSBCG_ERR_ARG;
    if (prm.poll_every < 1) prm.poll_every = 1;
    if (prm.x0 && !X) return DSBCG_ERR_ARG;
    const double dtol = prm.dtol > 0 ? prm.dtol : default_dtol(prec);
    const bool mixed = prec != P64;
    // true residuals, B and the accumulated solutions: FP64 fields for FP64
    // storage (or on request), double-float fields (FP32 arithmetic, 48-bit
    // significands) for the reduced storages; the m x m work likewise
    const int sfp64 = (!mixed || prm.fp64_residuals) ? 1 : 0;
    const int hp = sfp64 ? P64 : PDD;
    CKS(ensure_links(c, prec));
    CKS(ensure_links(c, hp));
    CKS(ensure_ws(c, m, s, prec, nbb));
    auto& w = c->ws;
    const size_t n = c->n, ld = c->ld;
    const size_t db = ld * sizeof(double2);
    for (int q = 0; q < 8; ++q) {
        c->kms[q] = 0;
        c->klaunch[q] = 0;
        c->kbytes[q] = 0;
        c->kflops[q] = 0;
    }

    // --- inputs: B -> internal high-precision fields (staging through X64's storage if on the host)
    const bool b_dev = is_device_ptr(B), x_dev = X && is_device_ptr(X);
    const size_t nb_fields = (size_t)nbb * m;
    double2* bcanon = nullptr;
    if (b_dev) {
        bcanon = (double2*)B;
    } else if (void* bmap = mapped_host_ptr(B)) {
        bcanon = (double2*)bmap;   // pinned and mapped: the kernels read it in place
    } else {
        bcanon = w.X64;        // X64 has >= nbb*m*ld complex; used as staging before it is zeroed
        CK(cudaMemcpyAsync(bcanon, B, nb_fields * n * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    }
    CK(cudaMemsetAsync(w.flag, 0, sizeof(int), c->st));
    {
        Prof p(c, DSBCG_KCLASS_OTHER, 2);
        launch_check_finite(bcanon, nb_fields * n, w.flag, c->st);
        pack_any(c, hp, w.B64, bcanon, (int)nb_fields);
    }
    int hflag = 0;
    CK(cudaMemcpyAsync(&hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemsetAsync(w.X64, 0, (size_t)s * m * db, c->st));
    // ||b_i||^2 via the residual kernel with x = 0 (A 0 = 0), per block of B
    std::vector<double> bn2(nb_fields), bn(nb_fields);
    {
        for (int jb = 0; jb < nbb; ++jb) {
            Prof p(c, DSBCG_KCLASS_OTHER, 2);
            const double2* bj = w.B64 + (size_t)jb * m * ld;
            if (hp == PDD)
                launch_residual_pairs((float2*)w.R64, (const float2*)bj, (const float2*)w.X64,
                                      (const float2*)w.X64, ld, m, n, 0.0, w.rpart, w.rblk, c->st);
            else
                launch_residual(w.R64, bj, w.X64, w.X64, ld, m, n, 0.0, w.rpart, w.rblk, c->st);
            launch_reduce_cols(w.rpart, w.rblk, m, w.norms + (size_t)jb * m, c->st);
        }
        CK(cudaMemcpyAsync(w.h_norms, w.norms, nb_fields * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (size_t i = 0; i < nb_fields; ++i) {
            bn2[i] = w.h_norms[i];
            bn[i] = sqrt(bn2[i]);
        }
    }
    // right-hand sides and their norms for shift j
    auto Bblk = [&](int j) { return w.B64 + (size_t)(nbb > 1 ? j : 0) * m * ld; };
    auto bnorm = [&](int j, int i) { return bn[(size_t)(nbb > 1 ? j : 0) * m + i]; };
    if (hflag) return DSBCG_ERR_NONFINITE;
    // --- initial guess (a resumed solve): X's input, packed shift by shift
    // into the high-precision X_j (the norms above were taken with X = 0)
    if (prm.x0) {
        const void* xin_map = x_dev ? nullptr : mapped_host_ptr(X);
        CK(cudaMemsetAsync(w.flag, 0, sizeof(int), c->st));
        for (int j = 0; j < s; ++j) {
            const double2* src = nullptr;
            if (x_dev) {
                src = (const double2*)X + (size_t)j * m * n;
            } else if (xin_map) {
                src = (const double2*)xin_map + (size_t)j * m * n;
            } else {
                CK(cudaMemcpyAsync(w.T64a, (const double2*)X + (size_t)j * m * n, (size_t)m * n * sizeof(double2),
                                   cudaMemcpyHostToDevice, c->st));
                src = w.T64a;
            }
            Prof p(c, DSBCG_KCLASS_OTHER, 2);
            launch_check_finite(src, (size_t)m * n, w.flag, c->st);
            pack_any(c, hp, w.X64 + (size_t)j * m * ld, src, m);
        }
        int xflag = 0;
        CK(cudaMemcpyAsync(&xflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (xflag) return DSBCG_ERR_NONFINITE;
    }

    std::vector<double> rel((size_t)s * m, 0.0);
    std::vector<int> conv((size_t)s * m, -1);
    std::vector<int> conv_tmp((size_t)s * m, -1);
    int total_steps = 0, restarts = 0, deflations = 0, final_rank = m;
    long long mvms = 0;
    dsbcg_status result = DSBCG_OK;
    // right-hand sides of the inner solves: the FP64 fields, or the FP32 hi
    // planes of the double-float fields
    const int rprec = hp == PDD ? P32 : P64;
    const size_t rld = hp_ld(c, hp);
    const double drop = mixed ? std::max(prm.restart_drop, 1e-12) : 0.0;
    // Inner solves aim at rt_frac x tol: each ends on its recurrence residual,
    // which the final FP64 true residual has to confirm below tol.  FP32 and
    // FP64 Krylov processes started from a true residual keep that estimate
    // within about 1e-3 of the starting residual (far below 0.1 tol here);
    // 16-bit processes drift more.  16^3 x 32 and 24^3 x 48 (m = 12 / 8) took
    // 341 / 763 ms at 0.9 against 354 / 792 at 0.5 in FP32 storage; BF16
    // needed extra restarts at 0.9 and was fastest at 0.7.
    const double rt_frac = (prec == PBF16 || prec == PF16) ? 0.7 : 0.9;

    // --- lanes for the per-shift restarts (allocated before the joint solve
    // starts, so that no allocation falls inside it).  With profiling on,
    // lane 0 alone on the context's stream (serial restarts, clean
    // per-kernel timings); results are bitwise the same.
    int lane_lo = 0, lane_hi = 1;                      // refinement lanes [lane_lo, lane_hi)
    if (prm.refine && !c->profiling && s > 1) {
        const int got = ensure_refine_lanes(c, 1 + std::min(s, 16));
        if (got > 1) {
            lane_lo = 1;
            lane_hi = got;
        }
    }
    // --- joint inner solve on B for all shifts (not with an initial guess or
    // per-shift right-hand sides: the shifts' residuals then differ, and each
    // is restarted on its own)
    // shifts whose X_j is still zero (per-shift right-hand sides): their
    // first residual is b itself, no operator application needed
    std::vector<char> xzero(s, (nbb > 1 && !prm.x0) ? 1 : 0);
    const bool joint = !prm.x0 && nbb == 1;
    // Early hand-off: a shift the joint solve has frozen (all its columns
    // below their targets; the shift update skips it from then on) has its
    // final inner iterate, so its true residual and restarts start while the
    // joint solve continues for the other shifts.  That work runs on the
    // refinement stream, and the restarts on their own lanes.
    const bool early = joint && prm.freeze_converged && lane_lo == 1;
    cudaStream_t fst = c->st;                          // residuals, gathers, accumulation, output
    if (early) {
        if (!c->rst) CK(cudaStreamCreateWithPriority(&c->rst, cudaStreamNonBlocking, stream_prio(true)));
        if (!c->ev_joint) CK(cudaEventCreateWithFlags(&c->ev_joint, cudaEventDisableTiming));
        if (!c->ev_ref) CK(cudaEventCreateWithFlags(&c->ev_ref, cudaEventDisableTiming));
        fst = c->rst;
    }
    // on every return: no work of this solve left in flight on the refinement
    // stream or the restart lanes (an error may leave lanes running)
    struct Quiesce {
        dsbcg_ctx* c;
        int lo, hi;
        ~Quiesce() {
            if (c->rst) cudaStreamSynchronize(c->rst);
            for (int l = lo; l < hi; ++l)
                if (c->ws.lanes[l].st != c->st) cudaStreamSynchronize(c->ws.lanes[l].st);
        }
    } quiesce{c, lane_lo, lane_hi};
    auto accumulate = [&](double2* y, const void* x, int nf) {
        Prof p(c, DSBCG_KCLASS_OTHER, 1, fst);
        if (hp == PDD)
            launch_accumulate_pairs((float2*)y, ld, (const float2*)x, ld, nf, n, fst);
        else
            launch_accumulate(work_prec(prec), y, ld, x, ld, nf, n, fst);
    };
    std::vector<int> conv_joint((size_t)s * m, -1);
    Lane* L0 = &w.lanes[0];
    bool joint_running = false;
    std::vector<char> handed(s, 0);
    std::deque<int> queue;
    // shift j's inner iterate is final: add it to X_j and queue its residual
    auto handoff = [&](int j) -> dsbcg_status {
        accumulate(w.X64 + (size_t)j * m * ld, (const char*)w.Xin + (size_t)j * m * ld * prec_elem_bytes(work_prec(prec)), m);
        handed[j] = 1;
        queue.push_back(j);
        return DSBCG_OK;
    };
    auto joint_done = [&]() -> dsbcg_status {
        InnerResult ir;
        CKS(lane_finish(c, *L0, &ir, 0, conv_joint.data()));
        joint_running = false;
        total_steps += ir.steps;
        mvms += ir.mvms;
        deflations += ir.deflations;
        final_rank = ir.final_rank;
        if (ir.status == DSBCG_ERR_NOT_HPD) return DSBCG_ERR_NOT_HPD;
        if (ir.status != 0) return DSBCG_ERR_CUDA;
        return DSBCG_OK;
    };
    if (joint) {
        Range r_joint("joint block solve");
        std::vector<double> tg((size_t)s * m);
        for (int j = 0; j < s; ++j)
            for (int i = 0; i < m; ++i) tg[(size_t)j * m + i] = std::max(drop * bn[i], rt_frac * tol * bn[i]);
        CKS(lane_start(c, *L0, w.B64, rprec, rld, m, sigma, s, tg.data(), prec, dtol, prm.max_block_steps,
                       prm.freeze_converged, prm.poll_every, sfp64));
        if (early) {
            // the refinement stream starts after everything the solve has
            // enqueued on the context's stream so far
            CK(cudaEventRecord(c->ev_joint, c->st));
            CK(cudaStreamWaitEvent(c->rst, c->ev_joint, 0));
            CKS(lane_enqueue(c, *L0));
            joint_running = true;
        } else {
            CKS(run_lanes(c, &L0, 1));
            CKS(joint_done());
            accumulate(w.X64, w.Xin, s * m);
            for (int j = 0; j < s; ++j) queue.push_back(j);
        }
    } else {
        for (int j = 0; j < s; ++j) queue.push_back(j);
    }
    // joint lane whose enqueued batch has drained: hand off the shifts it has
    // frozen and give it its next batch, or finish it and hand off the rest.
    // `polled` tells whether the batch had drained.
    auto service_joint = [&](bool* polled) -> dsbcg_status {
        *polled = false;
        if (!joint_running) return DSBCG_OK;
        const cudaError_t e = cudaStreamQuery(c->st);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            return DSBCG_OK;
        }
        CK(e);
        *polled = true;
        CKS(lane_poll(c, *L0));
        if (L0->running) {
            bool any = false;
            for (int j = 0; j < s; ++j) any |= !handed[j] && L0->h_active[j] == 0;
            if (any) {
                // the joint stream is idle here: the event orders the
                // refinement stream after its last batch
                CK(cudaEventRecord(c->ev_joint, c->st));
                CK(cudaStreamWaitEvent(fst, c->ev_joint, 0));
                for (int j = 0; j < s; ++j)
                    if (!handed[j] && L0->h_active[j] == 0) CKS(handoff(j));
            }
            CKS(lane_enqueue(c, *L0));
        } else {
            CKS(joint_done());
            CK(cudaEventRecord(c->ev_joint, c->st));
            CK(cudaStreamWaitEvent(fst, c->ev_joint, 0));
            for (int j = 0; j < s; ++j)
                if (!handed[j]) CKS(handoff(j));
        }
        return DSBCG_OK;
    };
    // block steps so far, the running joint solve's included
    auto steps_so_far = [&]() { return total_steps + (joint_running ? L0->step : 0); };
    // --- output of a finished shift: its X_j goes to the caller's buffer as
    // soon as its last true residual is in (device or mapped pinned host
    // memory; other host memory is staged at the end), so that the transfer
    // overlaps the restarts of the other shifts
    void* const xmap = (x_dev || !X) ? nullptr : mapped_host_ptr(X);
    double2* const xout = x_dev ? (double2*)X : (double2*)xmap;
    auto emit = [&](int j) {
        if (!xout) return;
        Prof p(c, DSBCG_KCLASS_OTHER, 1, fst);
        unpack_any(c, hp, xout + (size_t)j * m * n, w.X64 + (size_t)j * m * ld, m, fst);
    };
    // --- high-precision true residuals and per-shift restarts.  Each shift
    // has a list of unconverged columns (initially all) and waits in a queue
    // for its true residual, taken on the refinement stream.  Columns still
    // above tol become the right-hand sides of a restart of that shift (block
    // CG on sigma_j I + A) on a free lane; lanes run concurrently on their
    // own streams, and a finished restart's solution is added to X_j and the
    // shift queued again, so residuals overlap the restarts still running.
    std::vector<double> r2(m);
    std::vector<std::vector<int>> cols(s);
    std::vector<char> full(s, 1);           // residual of all m columns still to be taken
    std::vector<int> lane_j(w.lanes.size(), -1);       // shift restarted on each lane
    std::vector<std::vector<double>> lane_tg(w.lanes.size());
    auto gather = [&](double2* dst, const double2* src, const std::vector<int>& idx) -> dsbcg_status {
        for (size_t q = 0; q < idx.size(); ++q)
            CK(cudaMemcpyAsync(dst + q * ld, src + (size_t)idx[q] * ld, db, cudaMemcpyDeviceToDevice, fst));
        return DSBCG_OK;
    };
    // while the host waits for a true residual: keep the joint lane and
    // every running restart lane whose enqueued batch has drained supplied
    // (finished restart lanes are left to the main loop)
    const std::function<dsbcg_status()> service_lanes = [&]() -> dsbcg_status {
        bool polled;
        CKS(service_joint(&polled));
        for (int l = lane_lo; l < lane_hi; ++l) {
            Lane& L = w.lanes[l];
            if (lane_j[l] < 0 || L.st == c->st || !L.running) continue;
            const cudaError_t e = cudaStreamQuery(L.st);
            if (e == cudaErrorNotReady) {
                cudaGetLastError();
                continue;
            }
            CK(e);
            CKS(lane_poll(c, L));
            if (L.running) CKS(lane_enqueue(c, L));
        }
        return DSBCG_OK;
    };
    // residuals of queued shifts while a lane is free; restarts where needed
    auto feed = [&]() -> dsbcg_status {
        for (;;) {
            int li = -1;
            for (int l = lane_lo; l < lane_hi; ++l)
                if (lane_j[l] < 0) {
                    li = l;
                    break;
                }
            if (li < 0 || queue.empty()) return DSBCG_OK;
            const int j = queue.front();
            queue.pop_front();
            double2* Xj = w.X64 + (size_t)j * m * ld;
            std::vector<int>& cl = cols[j];
            if (full[j] && xzero[j]) {
                // X_j = 0: the residual is b_j itself
                cl.resize(m);
                for (int i = 0; i < m; ++i) {
                    cl[i] = i;
                    r2[i] = bnorm(j, i) * bnorm(j, i);
                }
                CK(cudaMemcpyAsync(w.R64, Bblk(j), (size_t)m * db, cudaMemcpyDeviceToDevice, fst));
                full[j] = 0;
                xzero[j] = 0;
            } else if (full[j]) {
                cl.resize(m);
                for (int i = 0; i < m; ++i) cl[i] = i;
                CKS(true_residual(c, hp, w.R64, Bblk(j), Xj, m, sigma[j], r2.data(), &service_lanes, fst));
                full[j] = 0;
                mvms += (long long)cl.size();
            } else {
                CKS(gather(w.Xg, Xj, cl));
                CKS(gather(w.Bg, Bblk(j), cl));
                CKS(true_residual(c, hp, w.R64, w.Bg, w.Xg, (int)cl.size(), sigma[j], r2.data(), &service_lanes, fst));
                mvms += (long long)cl.size();
            }
            std::vector<int> next, src;        // unconverged columns; their rows of R64
            for (size_t q = 0; q < cl.size(); ++q) {
                const int i = cl[q];
                const double bi = bnorm(j, i);
                rel[(size_t)j * m + i] = bi > 0 ? sqrt(r2[q]) / bi : 0.0;
                if (rel[(size_t)j * m + i] > tol) {
                    next.push_back(i);
                    src.push_back((int)q);
                }
            }
            cl.swap(next);
            if (cl.empty() || !prm.refine || restarts >= prm.max_restarts || steps_so_far() >= prm.max_block_steps) {
                emit(j);                        // X_j is final
                continue;
            }
            Lane& L = w.lanes[li];
            const int mu = (int)cl.size();
            std::vector<double>& tg = lane_tg[li];
            tg.resize(mu);
            for (int q = 0; q < mu; ++q) {
                const int i = cl[q];
                tg[q] = std::max(drop * rel[(size_t)j * m + i] * bnorm(j, i), rt_frac * tol * bnorm(j, i));
            }
            CKS(gather(L.rhs, w.R64, src));
            if (L.st != fst) {
                CK(cudaEventRecord(L.ready, fst));
                CK(cudaStreamWaitEvent(L.st, L.ready, 0));
            }
            CKS(lane_start(c, L, L.rhs, rprec, rld, mu, &sigma[j], 1, tg.data(), prec, dtol,
                           std::max(1, prm.max_block_steps - steps_so_far()), prm.freeze_converged, prm.poll_every,
                           sfp64));
            CKS(lane_enqueue(c, L));
            restarts += 1;
            lane_j[li] = j;
        }
    };
    Range r_ref("per-shift restarts");
    CKS(feed());
    for (;;) {
        bool busy = joint_running;
        for (int l = lane_lo; l < lane_hi; ++l)
            if (lane_j[l] >= 0) busy = true;
        if (!busy) break;
        // service the joint lane and the restart lanes whose enqueued batch
        // has drained, as soon as any has (non-blocking queries): a lane
        // never waits for the host to finish waiting on a slower lane
        std::vector<int> ready;
        for (long spins = 0;; ++spins) {
            bool polled = false;
            CKS(service_joint(&polled));
            for (int l = lane_lo; l < lane_hi; ++l) {
                if (lane_j[l] < 0) continue;
                const cudaError_t e = cudaStreamQuery(w.lanes[l].st);
                if (e == cudaSuccess) {
                    ready.push_back(l);
                } else if (e == cudaErrorNotReady) {
                    cudaGetLastError();
                } else {
                    CK(e);
                }
            }
            if (polled || !ready.empty()) break;
            if (spins > 64) std::this_thread::yield();
        }
        for (int l : ready) CKS(lane_poll(c, w.lanes[l]));
        prof_collect(c);
        for (int l : ready) {
            Lane& L = w.lanes[l];
            if (L.running) {
                CKS(lane_enqueue(c, L));
                continue;
            }
            // restart finished: fold its solution into X_j
            const int j = lane_j[l];
            InnerResult ir;
            CKS(lane_finish(c, L, &ir, steps_so_far(), conv_tmp.data()));
            total_steps += ir.steps;
            mvms += ir.mvms;
            deflations += ir.deflations;
            if (ir.status == DSBCG_ERR_NOT_HPD) return DSBCG_ERR_NOT_HPD;
            if (ir.status != 0) return DSBCG_ERR_CUDA;
            double2* Xj = w.X64 + (size_t)j * m * ld;
            for (size_t q = 0; q < cols[j].size(); ++q) {
                if (conv_tmp[q] >= 0) conv[(size_t)j * m + cols[j][q]] = conv_tmp[q];
                accumulate(Xj + (size_t)cols[j][q] * ld,
                           (char*)L.Xin + q * ld * prec_elem_bytes(work_prec(prec)), 1);
            }
            lane_j[l] = -1;
            queue.push_back(j);           // its new residual decides the next restart
        }
        CKS(feed());
    }
    // a column no restart reached keeps the step at which the joint solve
    // froze it
    for (size_t t = 0; t < conv.size(); ++t)
        if (conv[t] < 0) conv[t] = conv_joint[t];
    if (early) {
        // the output stage below runs on the context's stream
        CK(cudaEventRecord(c->ev_ref, c->rst));
        CK(cudaStreamWaitEvent(c->st, c->ev_ref, 0));
    }
    for (double r : rel)
        if (!(r <= tol)) result = DSBCG_NOT_CONVERGED;

    // --- output X (canonical complex128 [s][m][n]): device and mapped pinned
    // host buffers were written shift by shift above
    auto unpack = [&](double2* dst, const double2* src, int nf) {
        Prof p(c, DSBCG_KCLASS_OTHER);
        unpack_any(c, hp, dst, src, nf);
    };
    if (rat) {
        // Y = alpha_0 B + sum_j alpha_j X_j in one pass over the final
        // solutions, shifts summed in index order (bitwise reproducible)
        std::vector<double> coef(s + 1);
        coef[0] = rat->alpha0;
        for (int j = 0; j < s; ++j) coef[j + 1] = rat->alpha[j];
        CK(cudaMemcpyAsync(w.coefR, coef.data(), (s + 1) * sizeof(double), cudaMemcpyHostToDevice, c->st));
        const bool y_dev = is_device_ptr(rat->Y);
        void* ymap = y_dev ? nullptr : mapped_host_ptr(rat->Y);
        double2* ydst = y_dev ? (double2*)rat->Y : (ymap ? (double2*)ymap : w.T64a);
        {
            Prof p(c, DSBCG_KCLASS_OTHER);
            launch_rational_combine(hp, ydst, w.B64, w.X64, ld, m, s, w.coefR, c->Vf, c->st);
        }
        c->kbytes[DSBCG_KCLASS_OTHER] += (double)(s + 1) * m * n * 16.0 + (double)m * n * 16.0;
        if (!y_dev && !ymap)
            CK(cudaMemcpyAsync(rat->Y, w.T64a, (size_t)m * n * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
    }
    if (xout || !X) {
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(c->st));
    } else {
        // stage one shift at a time through R64/T64a (m fields each)
        for (int j = 0; j < s; ++j) {
            unpack(w.T64a, w.X64 + (size_t)j * m * ld, m);
            CK(cudaMemcpyAsync((double2*)X + (size_t)j * m * n, w.T64a, (size_t)m * n * sizeof(double2),
                               cudaMemcpyDeviceToHost, c->st));
        }
        CK(cudaStreamSynchronize(c->st));
    }
    prof_collect(c);
    if (stats) {
        stats->block_steps = total_steps;
        stats->mvms = mvms;
        stats->deflations = deflations;
        stats->restarts = restarts;
        stats->final_rank = final_rank;
        if (stats->true_relres) memcpy(stats->true_relres, rel.data(), rel.size() * sizeof(double));
        if (stats->conv_step) memcpy(stats->conv_step, conv.data(), conv.size() * sizeof(int));
        for (int q = 0; q < 8; ++q) {
            stats->kernel_ms[q] = c->kms[q];
            stats->kernel_launches[q] = c->klaunch[q];
            stats->kernel_bytes[q] = c->kbytes[q];
            stats->kernel_flops[q] = c->kflops[q];
        }
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return result;
}

}  // namespace


extern "C" {

void dsbcg_params_default(dsbcg_params* p) {
    if (!p) return;
    p->storage = DSBCG_PREC_FP32;
    p->dtol = 0.0;
    p->max_block_steps = 100000;
    p->max_restarts = 50;
    p->restart_drop = 1e-7;
    p->poll_every = 16;
    p->freeze_converged = 1;
    p->refine = 1;
    p->fp64_residuals = 1;
    p->x0 = 0;
}

const char* dsbcg_error_string(dsbcg_status s) {
    switch (s) {
        case DSBCG_OK: return "ok";
        case DSBCG_NOT_CONVERGED: return "not converged (iteration or restart cap reached)";
        case DSBCG_ERR_ARG: return "invalid argument";
        case DSBCG_ERR_NOT_HPD: return "sigma_j I + T is not hermitian positive definite";
        case DSBCG_ERR_CUDA: return "CUDA runtime error";
        case DSBCG_ERR_OOM: return "device out of memory";
        case DSBCG_ERR_NONFINITE: return "non-finite input";
        case DSBCG_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char* dsbcg_version(void) { return "dsbcg 0.1 sm_103a"; }

dsbcg_status dsbcg_create(dsbcg_ctx** out, const int dims[4], const void* gauge, double kappa, int t_antiperiodic,
                          void* stream) {
    if (!out || !dims || !gauge) return DSBCG_ERR_ARG;
    *out = nullptr;
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2 || dims[d] > 4096) return DSBCG_ERR_ARG;
    if (!(kappa == kappa) || !isfinite(kappa)) return DSBCG_ERR_ARG;
    size_t V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (size_t)1 << 30) return DSBCG_ERR_ARG;
    dsbcg_ctx* c = new dsbcg_ctx();
    for (int d = 0; d < 4; ++d) c->g.L[d] = dims[d];
    c->g.V = (int)V;
    c->g.tap = t_antiperiodic ? 1 : 0;
    c->V = V;
    c->Vf = V;
    c->n = 12 * V;
    c->ld = (c->n + 127) / 128 * 128;
    c->kappa = kappa;
    c->st = (cudaStream_t)stream;
    // 16-bit scale: power of two near sqrt(n)
    c->hscale = (float)ldexp(1.0, (int)lround(0.5 * log2((double)c->n)));
    dsbcg_status st = dsbcg_update_gauge(c, gauge);
    if (st != DSBCG_OK) {
        dsbcg_destroy(c);
        return st;
    }
    *out = c;
    return DSBCG_OK;
}

dsbcg_status dsbcg_update_gauge(dsbcg_ctx* c, const void* gauge) {
    if (!c || !gauge) return DSBCG_ERR_ARG;
    // From here until the new field has been checked and packed the context
    // holds no usable field: the old packed links go first, so that no
    // precision keeps links of the old field while gauge64 holds the new one.
    c->gauge_ok = false;
    c->su3 = false;
    for (int p = 0; p < 5; ++p) {
        if (c->links[p]) {
            cudaFree(c->links[p]);
            c->links[p] = nullptr;
        }
        if (c->links12[p]) {
            cudaFree(c->links12[p]);
            c->links12[p] = nullptr;
        }
    }
    const size_t bytes = c->V * 36 * sizeof(double2);
    if (!c->gauge64) CK(cudaMalloc((void**)&c->gauge64, bytes));
    CK(cudaMemcpyAsync(c->gauge64, gauge, bytes, is_device_ptr(gauge) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->st));
    int* flag = nullptr;
    CK(cudaMalloc((void**)&flag, 2 * sizeof(int)));
    cudaMemsetAsync(flag, 0, sizeof(int), c->st);
    launch_check_finite(c->gauge64, c->V * 36, flag, c->st);
    int h = 0;
    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    // a field in SU(3) to 1e-10 gets 12-real links for the reduced storages
    int hs = 1;
    cudaMemsetAsync(flag + 1, 0, sizeof(int), c->st);
    launch_check_su3(c->gauge64, c->V * 4, 1e-10, flag + 1, c->st);
    cudaMemcpyAsync(&hs, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    const cudaError_t e = cudaStreamSynchronize(c->st);
    cudaFree(flag);
    CK(e);
    if (h) return DSBCG_ERR_NONFINITE;
    c->su3 = (hs == 0);
    CKS(ensure_links(c, P64));
    c->gauge_ok = true;
    return DSBCG_OK;
}

dsbcg_status dsbcg_solve(dsbcg_ctx* c, int m, const void* B, int s, const double* sigma, double tol,
                         const dsbcg_params* params, void* X, dsbcg_stats* stats) {
    if (!X) return DSBCG_ERR_ARG;
    return solve_core(c, m, B, 1, s, sigma, tol, params, X, stats, nullptr);
}

dsbcg_status dsbcg_solve_rational(dsbcg_ctx* c, int m, const void* B, int s, const double* sigma, double alpha0,
                                  const double* alpha, double tol, const dsbcg_params* params, void* Y, void* X,
                                  dsbcg_stats* stats) {
    if (!Y || !alpha) return DSBCG_ERR_ARG;
    const RationalOut r{alpha0, alpha, Y};
    return solve_core(c, m, B, 1, s, sigma, tol, params, X, stats, &r);
}

void dsbcg_destroy(dsbcg_ctx* c) {
    if (!c) return;
    free_ws(c);
    for (int p = 0; p < 5; ++p) {
        if (c->links[p]) cudaFree(c->links[p]);
        if (c->links12[p]) cudaFree(c->links12[p]);
    }
    if (c->gauge64) cudaFree(c->gauge64);
    if (c->rst) cudaStreamDestroy(c->rst);
    if (c->ev_joint) cudaEventDestroy(c->ev_joint);
    if (c->ev_ref) cudaEventDestroy(c->ev_ref);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto& k : c->ev_live) {
        cudaEventDestroy(k.a);
        cudaEventDestroy(k.b);
    }
    delete c;
}

dsbcg_status dsbcg_debug_shift_chunk(dsbcg_ctx* c, int steps) {
    if (!c || steps < 0 || steps > CTL_HIST) return DSBCG_ERR_ARG;
    c->force_chunk = steps;
    return DSBCG_OK;
}

dsbcg_status dsbcg_debug_first_wait(dsbcg_ctx* c, int polls) {
    if (!c) return DSBCG_ERR_ARG;
    c->debug_first_wait = polls < 0 ? -1 : polls;
    return DSBCG_OK;
}

dsbcg_status dsbcg_set_profiling(dsbcg_ctx* c, int on) {
    if (!c) return DSBCG_ERR_ARG;
    c->profiling = on != 0;
    return DSBCG_OK;
}

dsbcg_status dsbcg_read_profile(dsbcg_ctx* c, double kernel_ms[8], long long kernel_launches[8]) {
    if (!c) return DSBCG_ERR_ARG;
    CK(cudaStreamSynchronize(c->st));
    prof_collect(c);
    for (int q = 0; q < 8; ++q) {
        if (kernel_ms) kernel_ms[q] = c->kms[q];
        if (kernel_launches) kernel_launches[q] = c->klaunch[q];
        c->kms[q] = 0;
        c->klaunch[q] = 0;
        c->kbytes[q] = 0;
        c->kflops[q] = 0;
    }
    return DSBCG_OK;
}

dsbcg_status dsbcg_apply(dsbcg_ctx* c, int op, int storage, int m, const void* in, void* out) {
    if (!c || !in || !out || m < 1 || m > 4096 || op < 0 || op > 2 || storage < 0 || storage > PDD)
        return DSBCG_ERR_ARG;
    if (!c->gauge_ok) return DSBCG_ERR_ARG;
    CKS(ensure_links(c, storage));
    const size_t n = c->n, ld = hp_ld(c, storage);
    const size_t fb = prec_elem_bytes(storage) * c->ld;
    void *a = nullptr, *b = nullptr, *t = nullptr, *t2 = nullptr;
    double2 *din = nullptr, *dout = nullptr;
    const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
    dsbcg_status rs = DSBCG_OK;
    auto fail = [&](dsbcg_status s) { rs = s; };
    if (cudaMalloc(&a, m * fb) != cudaSuccess || cudaMalloc(&b, m * fb) != cudaSuccess ||
        cudaMalloc(&t, m * fb) != cudaSuccess || (c->schur && cudaMalloc(&t2, m * fb) != cudaSuccess)) {
        fail(DSBCG_ERR_OOM);
    }
    if (rs == DSBCG_OK && !in_dev) {
        if (cudaMalloc((void**)&din, m * n * sizeof(double2)) != cudaSuccess) fail(DSBCG_ERR_OOM);
        else cudaMemcpyAsync(din, in, m * n * sizeof(double2), cudaMemcpyHostToDevice, c->st);
    }
    if (rs == DSBCG_OK && !out_dev) {
        if (cudaMalloc((void**)&dout, m * n * sizeof(double2)) != cudaSuccess) fail(DSBCG_ERR_OOM);
    }
    if (rs == DSBCG_OK) {
        const double2* src = in_dev ? (const double2*)in : din;
        double2* dst = out_dev ? (double2*)out : dout;
        pack_any(c, storage, a, src, m);
        if (op == DSBCG_OP_A) {
            apply_op(c, storage, b, t, a, t2, ld, nullptr, m, m, c->hscale, c->st, DSBCG_KCLASS_DSLASH);
        } else if (c->schur) {
            apply_dhat(c, storage, b, a, t, ld, op == DSBCG_OP_DDAG, nullptr, m, m, c->hscale, c->st,
                       DSBCG_KCLASS_DSLASH);
        } else {
            Prof p(c, DSBCG_KCLASS_DSLASH);
            launch_dslash(storage, b, a, ld, c->links[storage], c->g, c->kappa, op == DSBCG_OP_DDAG, nullptr, m, m,
                          c->hscale, c->st, c->links12[storage]);
        }
        unpack_any(c, storage, dst, b, m);
        if (!out_dev) cudaMemcpyAsync(out, dout, m * n * sizeof(double2), cudaMemcpyDeviceToHost, c->st);
        if (cudaGetLastError() != cudaSuccess) fail(DSBCG_ERR_CUDA);
        if (cudaStreamSynchronize(c->st) != cudaSuccess) fail(DSBCG_ERR_CUDA);
        prof_collect(c);
    }
    cudaFree(a);
    cudaFree(b);
    cudaFree(t);
    if (t2) cudaFree(t2);
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    return rs;
}

dsbcg_status dsbcg_set_operator(dsbcg_ctx* c, int op) {
    if (!c || (op != DSBCG_OPERATOR_NORMAL && op != DSBCG_OPERATOR_SCHUR)) return DSBCG_ERR_ARG;
    if (op == DSBCG_OPERATOR_SCHUR)
        for (int d = 0; d < 4; ++d)
            if (c->g.L[d] % 2) return DSBCG_ERR_ARG;
    if ((op == DSBCG_OPERATOR_SCHUR) == (c->schur != 0)) return DSBCG_OK;
    free_ws(c);                          // workspaces are sized for the field length
    c->schur = op == DSBCG_OPERATOR_SCHUR;
    c->Vf = c->schur ? c->V / 2 : c->V;
    c->n = 12 * c->Vf;
    c->ld = (c->n + 127) / 128 * 128;
    c->hscale = (float)ldexp(1.0, (int)lround(0.5 * log2((double)c->n)));
    return DSBCG_OK;
}

dsbcg_status dsbcg_force(dsbcg_ctx* c, int m, int s, const void* X, const void* Lambda, const double* weights,
                         int storage, void* dU) {
    if (!c || !X || !Lambda || !dU || m < 1 || s < 1 || (size_t)m * s > 4096) return DSBCG_ERR_ARG;
    if (!c->gauge_ok) return DSBCG_ERR_ARG;
    if (storage != P64 && storage != P32) return DSBCG_ERR_UNSUPPORTED;
    if (c->schur) return DSBCG_ERR_UNSUPPORTED;     // the force of the normal operator only
    CKS(ensure_links(c, storage));
    const size_t n = c->n, ld = c->ld, V = c->V;
    const int nf = m * s;
    const size_t fb = prec_elem_bytes(storage) * ld;
    const size_t cb = (size_t)nf * n * sizeof(double2);
    void *xf = nullptr, *lf = nullptr, *ex = nullptr, *el = nullptr;
    double2 *stage = nullptr, *du = nullptr;
    double* wf = nullptr;
    dsbcg_status rs = DSBCG_OK;
    if (cudaMalloc(&xf, nf * fb) || cudaMalloc(&lf, nf * fb) || cudaMalloc(&ex, nf * fb) ||
        cudaMalloc(&el, nf * fb) || cudaMalloc((void**)&du, V * 36 * sizeof(double2)) ||
        cudaMalloc((void**)&wf, nf * sizeof(double)))
        rs = DSBCG_ERR_OOM;
    const bool xd = is_device_ptr(X), ldv = is_device_ptr(Lambda), ud = is_device_ptr(dU);
    if (rs == DSBCG_OK && (!xd || !ldv)) {
        if (cudaMalloc((void**)&stage, cb)) rs = DSBCG_ERR_OOM;
    }
    if (rs == DSBCG_OK) {
        std::vector<double> wh(nf);
        for (int j = 0; j < s; ++j)
            for (int i = 0; i < m; ++i) wh[(size_t)j * m + i] = weights ? weights[j] : 1.0;
        cudaMemcpyAsync(wf, wh.data(), nf * sizeof(double), cudaMemcpyHostToDevice, c->st);
        const double2* xs = (const double2*)X;
        if (!xd) {
            cudaMemcpyAsync(stage, X, cb, cudaMemcpyHostToDevice, c->st);
            xs = stage;
        }
        launch_pack_fields(storage, xf, ld, xs, nf, V, 1.f, c->st);
        const double2* ls = (const double2*)Lambda;
        if (!ldv) {
            cudaMemcpyAsync(stage, Lambda, cb, cudaMemcpyHostToDevice, c->st);
            ls = stage;
        }
        launch_pack_fields(storage, lf, ld, ls, nf, V, 1.f, c->st);
        launch_dslash(storage, ex, xf, ld, c->links[storage], c->g, c->kappa, 0, nullptr, nf, std::min(nf, 16), 1.f,
                      c->st, c->links12[storage]);
        launch_dslash(storage, el, lf, ld, c->links[storage], c->g, c->kappa, 0, nullptr, nf, std::min(nf, 16), 1.f,
                      c->st, c->links12[storage]);
        {
            Prof p(c, DSBCG_KCLASS_OTHER);
            launch_force(storage, du, ex, lf, el, xf, ld, nf, wf, c->g, c->kappa, c->st);
        }
        if (ud) {
            cudaMemcpyAsync(dU, du, V * 36 * sizeof(double2), cudaMemcpyDeviceToDevice, c->st);
        } else {
            cudaMemcpyAsync(dU, du, V * 36 * sizeof(double2), cudaMemcpyDeviceToHost, c->st);
        }
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->st) != cudaSuccess) rs = DSBCG_ERR_CUDA;
        prof_collect(c);
    }
    cudaFree(xf);
    cudaFree(lf);
    cudaFree(ex);
    cudaFree(el);
    cudaFree(du);
    cudaFree(wf);
    if (stage) cudaFree(stage);
    return rs;
}

dsbcg_status dsbcg_backward(dsbcg_ctx* c, int m, const void* B, int s, const double* sigma, const void* X,
                            const void* G, const double* g_weights, double g_direct, double tol,
                            const dsbcg_params* params, void* gB, double* gsigma, void* gU, void* Lambda,
                            dsbcg_stats* stats) {
    Range r_bwd("dsbcg_backward");
    auto t0 = std::chrono::steady_clock::now();
    if (!c || !G || !sigma || m < 1 || m > M_MAX || s < 1 || s > S_MAX) return DSBCG_ERR_ARG;
    if (!X && !B) return DSBCG_ERR_ARG;
    if (!c->gauge_ok) return DSBCG_ERR_ARG;
    if (gU && c->schur) return DSBCG_ERR_UNSUPPORTED;
    if (g_weights)
        for (int j = 0; j < s; ++j)
            if (!isfinite(g_weights[j])) return DSBCG_ERR_ARG;
    if (!isfinite(g_direct) || (g_direct != 0.0 && !g_weights)) return DSBCG_ERR_ARG;
    dsbcg_params prm;
    if (params) prm = *params;
    else dsbcg_params_default(&prm);
    prm.x0 = 0;
    const size_t n = c->n;
    const size_t cnt = (size_t)m * n, blk = (size_t)s * cnt;
    // X is needed by the shift gradient and the force only
    const bool need_x = gsigma || gU;
    std::vector<void*> owned;
    auto dalloc = [&](void** p, size_t bytes) -> dsbcg_status {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return DSBCG_ERR_OOM;
        }
        owned.push_back(*p);
        return DSBCG_OK;
    };
    dsbcg_status rs = DSBCG_OK, solve_st = DSBCG_OK;
    int steps = 0, restarts = 0, deflations = 0, final_rank = 0;
    long long mvms = 0;
    auto add_stats = [&](const dsbcg_stats& q) {
        steps += q.block_steps;
        mvms += q.mvms;
        deflations += q.deflations;
        restarts += q.restarts;
        final_rank = q.final_rank;
    };
    auto run = [&]() -> dsbcg_status {
        double2* Xd = nullptr;
        if (need_x) {
            if (X && is_device_ptr(X)) {
                Xd = (double2*)X;
            } else {
                CKS(dalloc((void**)&Xd, blk * sizeof(double2)));
                if (X) {
                    CK(cudaMemcpyAsync(Xd, X, blk * sizeof(double2), cudaMemcpyHostToDevice, c->st));
                } else {
                    // recompute the solutions instead of keeping them (memory)
                    dsbcg_stats q{};
                    const dsbcg_status st = solve_core(c, m, B, 1, s, sigma, tol, &prm, Xd, &q, nullptr);
                    if (st < 0) return st;
                    if (st == DSBCG_NOT_CONVERGED) solve_st = st;
                    add_stats(q);
                }
            }
        }
        // adjoint solves (sigma_j I + A) Lambda_j = G_j (sigma_j I + A is hermitian)
        double2* Ld = nullptr;
        if (Lambda && is_device_ptr(Lambda)) Ld = (double2*)Lambda;
        else CKS(dalloc((void**)&Ld, blk * sizeof(double2)));
        {
            dsbcg_stats q{};
            q.true_relres = stats ? stats->true_relres : nullptr;
            q.conv_step = stats ? stats->conv_step : nullptr;
            // one block with per-shift weights: one joint DSBlockCG solve, then
            // Lambda_j = w_j (sigma_j + A)^{-1} G; per-shift blocks: all shifts
            // in one call, each on its own refinement lane
            const dsbcg_status st = g_weights ? solve_core(c, m, G, 1, s, sigma, tol, &prm, Ld, &q, nullptr)
                                              : solve_core(c, m, G, s, s, sigma, tol, &prm, Ld, &q, nullptr);
            if (st < 0) return st;
            if (st == DSBCG_NOT_CONVERGED) solve_st = st;
            add_stats(q);
        }
        if (g_weights) {
            Prof p(c, DSBCG_KCLASS_OTHER);
            launch_scale_blocks(Ld, s, cnt, g_weights, c->st);
        }
        // dL/dB = g_direct G + sum_j Lambda_j
        if (gB) {
            const bool dev = is_device_ptr(gB);
            double2* dst = (double2*)gB;
            if (!dev) CKS(dalloc((void**)&dst, cnt * sizeof(double2)));
            const double2* gdev = (const double2*)G;
            if (g_direct != 0.0 && !is_device_ptr(G)) {
                double2* t = nullptr;
                CKS(dalloc((void**)&t, cnt * sizeof(double2)));
                CK(cudaMemcpyAsync(t, G, cnt * sizeof(double2), cudaMemcpyHostToDevice, c->st));
                gdev = t;
            }
            {
                Prof p(c, DSBCG_KCLASS_OTHER);
                launch_sum_blocks(dst, Ld, s, cnt, gdev, g_direct, c->st);
            }
            if (!dev) CK(cudaMemcpyAsync(gB, dst, cnt * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
        }
        // dL/dsigma_j = -Re tr(Lambda_j^H X_j)
        if (gsigma) {
            const int nblk = residual_blocks(cnt);
            double* part = nullptr;
            double* out = nullptr;
            CKS(dalloc((void**)&part, (size_t)nblk * s * sizeof(double)));
            CKS(dalloc((void**)&out, (size_t)s * sizeof(double)));
            {
                Prof p(c, DSBCG_KCLASS_OTHER, 2);
                launch_dot_re_blocks(Ld, Xd, s, cnt, part, nblk, out, c->st);
            }
            std::vector<double> h(s);
            CK(cudaMemcpyAsync(h.data(), out, s * sizeof(double), cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            for (int j = 0; j < s; ++j) gsigma[j] = -h[j];
        }
        // dL/dU: the force kernel over (X_j, Lambda_j)
        if (gU) CKS(dsbcg_force(c, m, s, Xd, Ld, nullptr, prm.storage == DSBCG_PREC_FP64 ? P64 : P32, gU));
        if (Lambda && (void*)Ld != Lambda)
            CK(cudaMemcpyAsync(Lambda, Ld, blk * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(c->st));
        return DSBCG_OK;
    };
    rs = run();
    cudaStreamSynchronize(c->st);
    for (void* p : owned) cudaFree(p);
    if (stats) {
        stats->block_steps = steps;
        stats->mvms = mvms;
        stats->deflations = deflations;
        stats->restarts = restarts;
        stats->final_rank = final_rank;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return rs != DSBCG_OK ? rs : solve_st;
}

}  // extern "C"

// ============================================================================
// dsbcg_apply_static: dsbcg_apply with its working fields in a static device
// array instead of cudaMalloc'd buffers (see include/dsbcg.h).
static __device__ __align__(256) unsigned char g_apply_scratch[DSBCG_STATIC_SCRATCH_BYTES];

namespace {

// Device address of g_apply_scratch on the current device, looked up once per
// device (host code may not use the symbol itself as a device pointer).
dsbcg_status static_scratch_address(void** out) {
    static std::mutex mu;
    static void* addr[128] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return DSBCG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return DSBCG_ERR_CUDA;
        }
        addr[dev] = p;
    }
    *out = addr[dev];
    return DSBCG_OK;
}

}  // namespace

extern "C" dsbcg_status dsbcg_apply_static(dsbcg_ctx* c, int op, int storage, int m, const void* in, void* out) {
    if (!c || !in || !out || m < 1 || op < 0 || op > 2 || storage < 0 || storage > PDD) return DSBCG_ERR_ARG;
    if (!c->gauge_ok) return DSBCG_ERR_ARG;
    if (!is_device_ptr(in) || !is_device_ptr(out)) return DSBCG_ERR_ARG;
    if (!c->links[storage] || c->schur) return DSBCG_ERR_UNSUPPORTED;
    const size_t ld = hp_ld(c, storage);
    const size_t fb = prec_elem_bytes(storage) * c->ld;
    const size_t nbuf = op == DSBCG_OP_A ? 3 : 2;
    if ((size_t)m > (size_t)DSBCG_STATIC_SCRATCH_BYTES / (nbuf * fb)) return DSBCG_ERR_ARG;
    void* base = nullptr;
    CKS(static_scratch_address(&base));
    char* a = (char*)base;
    char* b = a + (size_t)m * fb;
    char* t = b + (size_t)m * fb;
    const double2* src = (const double2*)in;
    double2* dst = (double2*)out;
    pack_any(c, storage, a, src, m);
    if (op == DSBCG_OP_D) {
        launch_dslash(storage, b, a, ld, c->links[storage], c->g, c->kappa, 0, nullptr, m, m, c->hscale, c->st);
    } else if (op == DSBCG_OP_DDAG) {
        launch_dslash(storage, b, a, ld, c->links[storage], c->g, c->kappa, 1, nullptr, m, m, c->hscale, c->st);
    } else {
        launch_dslash(storage, t, a, ld, c->links[storage], c->g, c->kappa, 0, nullptr, m, m, c->hscale, c->st);
        launch_dslash(storage, b, t, ld, c->links[storage], c->g, c->kappa, 1, nullptr, m, m, c->hscale, c->st);
    }
    unpack_any(c, storage, dst, b, m);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    return DSBCG_OK;
}
