// api.cu -- the C ABI of include/ppca.h: handle, validation, orchestration.
//
// Algorithm 1 (primed PCA) maps onto the calls as follows:
//   step 1 PRIMING            ppca_prime / ppca_prime_continue
//   steps 2-5 span, project,  ppca_finalize: Q = orth(V); G = (X Q)^T (X Q) in
//   full-PCA, return          one pass (on the CUDA-core engine and for FP8 data
//                             without a refine copy: Z = X^T X Q, G = Q^T Z);
//                             G = U diag(w) U^T; E = Q U[:, :k]; lambda = w / n
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "grouped.h"
#include "kernels.h"
#include "pass_tc.h"
#include "tc_host.h"

using namespace ppca;

namespace {
std::atomic<int64_t> g_launches{0};
}

void ppca::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t ppca::launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

namespace {

thread_local std::string g_last_error;

ppca_status fail(ppca_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define CUDA_TRY(expr)                                                                                   \
    do {                                                                                                 \
        cudaError_t e__ = (expr);                                                                        \
        if (e__ != cudaSuccess) return fail(PPCA_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), \
                                            __FILE__, __LINE__);                                         \
    } while (0)

#define PPCA_TRY(expr)                        \
    do {                                      \
        ppca_status s__ = (expr);             \
        if (s__ != PPCA_OK) return s__;       \
    } while (0)

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

int dtype_size(ppca_dtype t) { return t == PPCA_F32 ? 4 : (t == PPCA_BF16 ? 2 : 1); }

}  // namespace

ppca_status check_status_word(int* status);

struct ppca_handle {
    XView x;                  // data used by the priming passes
    XView xref;               // optional finalize copy
    bool has_ref = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int64_t ws_limit = 0;

    // workspace (sized for ws_m, ws_rows)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int ws_m = 0;
    int* status = nullptr;    // device status word (own 256-byte allocation; status[1] is the
                              // CholeskyQR fallback flag, status[2] the need for a second pass)

    float* V = nullptr;       // primed basis d x m
    float* Z = nullptr;       // pass output d x m
    float* Q = nullptr;       // orthonormal basis d x m (finalize)
    float* T = nullptr;       // temporary d x m
    float* buf = nullptr;     // EigenGame momentum d x m
    double* G = nullptr;      // m x m
    float* Rf = nullptr;      // m x m
    float* Gf = nullptr;      // m x m, FP32 copy of G (CholeskyQR's FP32 attempt)
    double* w = nullptr;      // m
    double* U = nullptr;      // m x m
    float* E_res = nullptr;   // d x m: ppca_finalize_host's eigenvectors before the copy out
    double* lam_res = nullptr;  // m: ppca_finalize_host's eigenvalues
    int* tile_rows = nullptr;   // ceil(n / 128): first rows of the blocks of a row sample
    double* seq_diff = nullptr; // POWER_SEQ: |x_t - x_{t+1}| of the last step; [1]: the row count
                                // summed across ranks (row sharding; the slot holds 256 bytes)
    float* gram_part = nullptr;
    void* jac = nullptr;
    double* eg = nullptr;
    SimtPassScratch simt;
    TcPassScratch tc;
    TcSchedule sched;

    // priming state
    int method = -1;
    int m = 0;
    int64_t t = 0;            // next minibatch step
    int64_t iters = 0;        // power iterations done
    ppca_prime_params params{};

    // row sharding: sum across ranks (NULL: one process), its context and staging buffer, rows of all ranks
    ppca_allreduce_fn ar_fn = nullptr;
    void* ar_ctx = nullptr;
    void* ar_stage = nullptr;
    int64_t ar_stage_bytes = 0;
    int64_t n_total = 0;

    // minibatch steps (Oja, EigenGame) replayed from a CUDA graph of kStepGraph
    // steps, captured once per shape and parameters (step_graphs)
    bool step_graphs = true;
    PrimerStep* pstep = nullptr;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[160] = {};

    // measurement
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    std::vector<int> event_prec;
    size_t events_used = 0;
    int64_t timed_passes[3] = {0, 0, 0}, timed_rows[3] = {0, 0, 0}, launch_base = 0;
};

namespace {

// Workspace for problems up to n x d with up to m directions (a batch slot
// sizes it for the largest instance it runs).
ppca_status ensure_workspace_dims(ppca_handle* h, int64_t n, int64_t d, int m) {
    if (h->ws && h->ws_m >= m) return PPCA_OK;
    const size_t dm = al256((size_t)d * m * sizeof(float));
    const int nsplit = simt_pass_nsplit(n, d, m, h->num_sms);
    size_t need = 5 * dm + al256((size_t)m * m * 8) + 2 * al256((size_t)m * m * 4) + al256((size_t)m * 8) +
                  al256((size_t)m * m * 8) + al256(gram_part_floats(d, m) * 4) + al256(jacobi_scratch_bytes(m)) +
                  dm + al256((size_t)m * 8) + al256((size_t)((n + 127) / 128) * 4) + al256(8) +
                  al256(sizeof(PrimerStep)) +
                  al256(eigengame_scratch_bytes(d, m)) + al256(simt_pass_scratch_floats(n, d, m, nsplit) * 4) +
                  al256(tc_pass_scratch_bytes(n, d, m, h->num_sms));
    if (h->ws_limit > 0 && (int64_t)need > h->ws_limit)
        return fail(PPCA_ERR_OOM, "workspace of %zu bytes exceeds the limit of %lld bytes", need,
                    (long long)h->ws_limit);
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
        h->ws = nullptr;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PPCA_ERR_OOM, "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
    }
    h->ws = p;
    h->ws_bytes = need;
    h->ws_m = m;
    char* c = static_cast<char*>(p);
    auto take = [&](size_t b) { char* r = c; c += al256(b); return r; };
    h->V = reinterpret_cast<float*>(take((size_t)d * m * 4));
    h->Z = reinterpret_cast<float*>(take((size_t)d * m * 4));
    h->Q = reinterpret_cast<float*>(take((size_t)d * m * 4));
    h->T = reinterpret_cast<float*>(take((size_t)d * m * 4));
    h->buf = reinterpret_cast<float*>(take((size_t)d * m * 4));
    h->G = reinterpret_cast<double*>(take((size_t)m * m * 8));
    h->Rf = reinterpret_cast<float*>(take((size_t)m * m * 4));
    h->Gf = reinterpret_cast<float*>(take((size_t)m * m * 4));
    h->w = reinterpret_cast<double*>(take((size_t)m * 8));
    h->U = reinterpret_cast<double*>(take((size_t)m * m * 8));
    h->E_res = reinterpret_cast<float*>(take((size_t)d * m * 4));
    h->lam_res = reinterpret_cast<double*>(take((size_t)m * 8));
    h->tile_rows = reinterpret_cast<int*>(take((size_t)((n + 127) / 128) * 4));
    h->seq_diff = reinterpret_cast<double*>(take(8));
    h->pstep = reinterpret_cast<PrimerStep*>(take(sizeof(PrimerStep)));
    h->gram_part = reinterpret_cast<float*>(take(gram_part_floats(d, m) * 4));
    h->jac = take(jacobi_scratch_bytes(m));
    h->eg = reinterpret_cast<double*>(take(eigengame_scratch_bytes(d, m)));
    h->simt.nsplit = nsplit;
    h->simt.Y = reinterpret_cast<float*>(take(simt_pass_scratch_floats(n, d, m, nsplit) * 4));
    h->simt.Zpart = h->simt.Y + (size_t)n * m;
    h->simt.zpart_floats = (int64_t)nsplit * d * m * 2;
    h->simt.num_sms = h->num_sms;
    h->tc = tc_pass_scratch_carve(take(tc_pass_scratch_bytes(n, d, m, h->num_sms)), n, d, m, h->num_sms);
    return PPCA_OK;
}

ppca_status ensure_workspace(ppca_handle* h, int m) { return ensure_workspace_dims(h, h->x.n, h->x.d, m); }

ppca_status validate_x(const void* X, int64_t n, int64_t d, int64_t ld, ppca_dtype dt, const float* scales) {
    if (!X) return fail(PPCA_ERR_INVALID, "X is NULL");
    if (n < 2) return fail(PPCA_ERR_INVALID, "n = %lld: need at least 2 points", (long long)n);
    if (d < 1) return fail(PPCA_ERR_INVALID, "d = %lld: need d >= 1", (long long)d);
    if (ld < d) return fail(PPCA_ERR_INVALID, "ld = %lld < d = %lld", (long long)ld, (long long)d);
    if (dt != PPCA_F32 && dt != PPCA_BF16 && dt != PPCA_FP8_E4M3) return fail(PPCA_ERR_INVALID, "unknown dtype %d", (int)dt);
    if ((dt == PPCA_FP8_E4M3) != (scales != nullptr))
        return fail(PPCA_ERR_INVALID, "row_scales must be given for FP8 data and only for FP8 data");
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return fail(PPCA_ERR_INVALID, "X is not 16-byte aligned");
    if ((ld * dtype_size(dt)) % 16 != 0)
        return fail(PPCA_ERR_INVALID, "row pitch ld * sizeof = %lld bytes is not a multiple of 16",
                    (long long)(ld * dtype_size(dt)));
    return PPCA_OK;
}

// Timing of one pass over rows [r0, r1): records the start event and returns
// the end event to record after the pass (nullptr when timing is off).
ppca_status pass_timer(ppca_handle* h, ppca_precision prec, int64_t rows, cudaEvent_t* ev_end) {
    *ev_end = nullptr;
    if (h->timing) {
        if (h->events_used == h->events.size()) {
            cudaEvent_t a, b;
            CUDA_TRY(cudaEventCreate(&a));
            CUDA_TRY(cudaEventCreate(&b));
            h->events.emplace_back(a, b);
            h->event_prec.push_back(0);
        }
        h->event_prec[h->events_used] = (int)prec;
        auto& pr = h->events[h->events_used++];
        CUDA_TRY(cudaEventRecord(pr.first, h->stream));
        *ev_end = pr.second;
        ++h->timed_passes[(int)prec];
        h->timed_rows[(int)prec] += rows;
    }
    return PPCA_OK;
}

// One X-pass over rows [r0, r1) of view x: Z = X^T X V.
ppca_status run_xpass(ppca_handle* h, const XView& x, const float* V, int m, int64_t r0, int64_t r1, float* Z,
                      ppca_precision prec) {
    cudaEvent_t ev_end = nullptr;
    PPCA_TRY(pass_timer(h, prec, r1 - r0, &ev_end));
    // FP32 data: 3xTF32 tensor cores for FAST passes; an ACCURATE X-pass (used
    // when priming is asked to run at full precision) runs on CUDA cores in
    // exact FP32 with double-float folding.  The pPCA step itself uses the
    // projected Gram (run_gram), which is accurate on tensor cores.
    const bool tc = h->sched.engine == 2 ? false
                    : h->sched.engine == 1 ? tc_pass_supported(x, m)
                                           : tc_pass_supported(x, m) && !(x.dtype == PPCA_F32 && prec == PPCA_PREC_ACCURATE);
    if (tc) {
        CUDA_TRY(xpass_tc(x, V, m, r0, r1, Z, prec, h->tc, h->sched, h->status, h->num_sms, h->stream));
    } else {
        CUDA_TRY(xpass_simt(x, V, m, r0, r1, Z, h->simt, h->stream));
    }
    if (ev_end) CUDA_TRY(cudaEventRecord(ev_end, h->stream));
    return PPCA_OK;
}

// Projected Gram over rows [r0, r1) of view x: G = (X Q)^T (X Q), FP64.
// Tensor cores for BF16 and FP32 data (one contraction, split precision);
// FP8 data (normally refined through a BF16/FP32 copy) and the CUDA-core
// engine: the exact-FP32 pass Z = X^T X Q, then G = Q^T Z in double-float.
ppca_status run_gram(ppca_handle* h, const XView& x, const float* Q, int m, int64_t r0, int64_t r1, double* G,
                     ppca_precision prec) {
    cudaEvent_t ev_end = nullptr;
    PPCA_TRY(pass_timer(h, prec, r1 - r0, &ev_end));
    if (tc_pass_supported(x, m) && x.dtype != PPCA_FP8_E4M3 && h->sched.engine != 2) {
        CUDA_TRY(projected_gram_tc(x, Q, m, r0, r1, G, prec, h->sched.flush, h->tc, h->status, h->num_sms,
                                   h->stream));
    } else {
        CUDA_TRY(xpass_simt(x, Q, m, r0, r1, h->T, h->simt, h->stream));
        CUDA_TRY(gram_df(Q, h->T, x.d, m, G, h->gram_part, h->stream));
    }
    if (ev_end) CUDA_TRY(cudaEventRecord(ev_end, h->stream));
    return PPCA_OK;
}

// CholeskyQR2: Q = orth(V) with positive diagonal, Q may alias V (the first
// pass writes the workspace buffer T, the second writes Q).  Both Gram
// matrices are accumulated in double-float.  The first Cholesky runs in FP32
// on the diagonally scaled Gram matrix and falls back to double-float on the
// device when its conditioning bound says V is too ill-conditioned for that;
// the second factors a matrix within rounding of the identity, in FP32.
// Row sharding: sum `count` elements (elem_bytes 4 or 8) of the device buffer
// buf over the ranks, through the caller's staging buffer when one was given.
ppca_status allreduce(ppca_handle* h, void* buf, int64_t count, int32_t elem_bytes) {
    if (!h->ar_fn) return PPCA_OK;
    const size_t bytes = (size_t)count * (size_t)elem_bytes;
    void* target = buf;
    if (h->ar_stage) {
        if ((int64_t)bytes > h->ar_stage_bytes)
            return fail(PPCA_ERR_INVALID, "all-reduce of %zu bytes exceeds the %lld-byte staging buffer", bytes,
                        (long long)h->ar_stage_bytes);
        CUDA_TRY(cudaMemcpyAsync(h->ar_stage, buf, bytes, cudaMemcpyDeviceToDevice, h->stream));
        target = h->ar_stage;
    }
    const ppca_status s = h->ar_fn(target, count, elem_bytes, h->stream, h->ar_ctx);
    if (s != PPCA_OK) return fail(s, "the all-reduce across ranks returned status %d", (int)s);
    if (h->ar_stage) CUDA_TRY(cudaMemcpyAsync(buf, h->ar_stage, bytes, cudaMemcpyDeviceToDevice, h->stream));
    return PPCA_OK;
}

// Rows of a minibatch (or a row sample) over all ranks: the local count, summed
// across ranks when the rows are sharded (one host read-back).
ppca_status global_rows(ppca_handle* h, int64_t local, int64_t* out) {
    *out = local;
    if (!h->ar_fn) return PPCA_OK;
    double v = (double)local;
    double* dev = h->seq_diff + 1;
    CUDA_TRY(cudaMemcpyAsync(dev, &v, sizeof v, cudaMemcpyHostToDevice, h->stream));
    PPCA_TRY(allreduce(h, dev, 1, 8));
    CUDA_TRY(cudaMemcpyAsync(&v, dev, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *out = (int64_t)(v + 0.5);
    return PPCA_OK;
}

int64_t rows_total(const ppca_handle* h) { return h->ar_fn ? h->n_total : h->x.n; }

// span_only: the caller needs span(Q) and a well-conditioned Q, not Q^T Q = I to
// working precision (a block power step: the next product and CholeskyQR see
// only the span).  Then, when the first pass's FP32 factor was accepted with a
// conditioning bound of at most 2^10 (Q^T Q within ~1e-4 of I), the second
// pass's Gram and factor are skipped on the device (R^-1 = I, Q = the first
// pass's result).
ppca_status run_orth(ppca_handle* h, const float* V, float* Q, int m, bool span_only = false) {
    const int64_t d = h->x.d;
    const float* src = V;
    // Tall bases (d >= 16384): Gram matrices on the tensor cores (three BF16
    // pieces, ~2^-24), which the FP32 factorisation cannot tell from exact; the
    // double-float fallback then recomputes its Gram in double-float (gated on
    // the rejection flag).  Shorter bases: the CUDA-core double-float Gram (the
    // two break even near d = 4096; at 262144 x 64 the tensor cores halve CholeskyQR2).
    const bool tc_gram = d >= 16384 && encode_fn() != nullptr && h->sched.engine != 2;
    const bool gate = span_only && !tc_gram;
    int* need_second = h->status + 2;            // device flag of the gated second pass
    for (int rep = 0; rep < 2; ++rep) {
        float* dst = rep == 0 ? h->T : Q;
        const int* run_if = gate && rep == 1 ? need_second : nullptr;
        if (tc_gram)
            CUDA_TRY(gram_tc(src, d, m, h->G, h->Gf, h->tc, h->status, h->num_sms, h->stream));
        else
            CUDA_TRY(gram_df(src, src, d, m, h->G, h->gram_part, h->stream, h->Gf, run_if));
        CUDA_TRY(cholesky_adaptive(h->G, h->Gf, m, h->Rf, rep == 0, h->status + 1, h->status, h->stream,
                                   tc_gram ? src : nullptr, d, h->gram_part,
                                   gate && rep == 0 ? need_second : nullptr, run_if));
        CUDA_TRY(apply_rinv(src, h->Rf, d, m, dst, h->stream));
        src = dst;
    }
    return PPCA_OK;
}

void minibatch(int64_t t, int64_t n, int64_t b, int64_t& r0, int64_t& r1) {
    const int64_t per_epoch = (n + b - 1) / b;
    const int64_t j = t % per_epoch;
    r0 = j * b;
    r1 = r0 + b < n ? r0 + b : n;
}

ppca_precision prime_prec(const ppca_handle* h) {
    const int p = h->params.precision;
    return p == PPCA_PREC_AUTO ? PPCA_PREC_FAST : (ppca_precision)p;
}

// The power method of Section 2.1, one direction at a time (T: step cap per
// direction).  Each step is one X-pass of the direction, then its projection
// on the complement of the directions found, normalisation and the distance to
// the previous iterate (power_seq_update, FP64), which is read back for the
// stopping test.
ppca_status run_power_seq(ppca_handle* h, int64_t T) {
    const int m = h->m;
    const int64_t n = h->x.n, d = h->x.d;
    const double eps = h->params.eps;
    for (int j = 0; j < m; ++j) {
        float* x = h->V + (size_t)j * d;
        for (int64_t t = 0; t < T; ++t) {
            PPCA_TRY(run_xpass(h, h->x, x, 1, 0, n, h->Z, prime_prec(h)));      // y = X^T X x
            PPCA_TRY(allreduce(h, h->Z, d, 4));
            CUDA_TRY(power_seq_update(h->V, d, j, h->Z, h->seq_diff, h->stream));
            ++h->iters;
            double diff = 0.0;
            CUDA_TRY(cudaMemcpyAsync(&diff, h->seq_diff, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CUDA_TRY(cudaStreamSynchronize(h->stream));
            if (diff < eps) break;
        }
    }
    return PPCA_OK;
}

// One minibatch step of Oja or EigenGame with host-side parameters.
ppca_status minibatch_step(ppca_handle* h) {
    const int m = h->m;
    const int64_t n = h->x.n, d = h->x.d;
    int64_t r0, r1;
    minibatch(h->t, n, h->params.batch, r0, r1);
    PPCA_TRY(run_xpass(h, h->x, h->V, m, r0, r1, h->Z, prime_prec(h)));
    PPCA_TRY(allreduce(h, h->Z, d * m, 4));                                       // the batch of all ranks
    int64_t b = 0;
    PPCA_TRY(global_rows(h, r1 - r0, &b));
    if (h->method == PPCA_OJA) {
        CUDA_TRY(gram_df(h->V, h->Z, d, m, h->G, h->gram_part, h->stream));       // S = Y^T Y = W^T Z
        const double lr = h->params.lr / ((double)h->t + h->params.lr_offset);
        CUDA_TRY(oja_update(h->V, h->Z, h->G, d, m, lr / (double)b, h->stream));
    } else {
        CUDA_TRY(gram_df(h->V, h->Z, d, m, h->G, h->gram_part, h->stream));       // C = V^T Z
        CUDA_TRY(eigengame_update(h->V, h->buf, h->Z, h->G, d, m, 1.0 / (double)b, h->params.lr,
                                  h->params.momentum, h->eg, h->stream));
    }
    ++h->t;
    return PPCA_OK;
}

// Graph-replayed steps.  Full minibatches of one epoch differ only in their
// first row (and Oja in its step size), so a step whose kernels read those
// from the device state (primer_step_begin) is the same for every t: a CUDA
// graph of kStepGraph such steps is captured once and replayed, saving the
// launch gaps of its ~10 small kernels per step.  The kernels and their
// arithmetic are those of minibatch_step: the results are the same bits.
constexpr int kStepGraph = 16;

struct StepGraphKey {
    int method, m, dtype, prec;
    int64_t n, d, ld, batch;
    const void* x;
    const void* ws;
    double lr, lr_offset, momentum;
    TcSchedule sched;
};

bool step_graph_eligible(const ppca_handle* h) {
    if (!h->step_graphs || h->ar_fn || h->timing) return false;
    // the caller is capturing the handle's stream: plain steps, which it can capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cap != cudaStreamCaptureStatusNone) return false;
    if (h->method != PPCA_OJA && h->method != PPCA_EIGENGAME) return false;
    const ppca_precision prec = prime_prec(h);
    const bool supported = tc_pass_supported(h->x, h->m);
    const bool tc = h->sched.engine == 2 ? false
                    : h->sched.engine == 1 ? supported
                                           : supported && !(h->x.dtype == PPCA_F32 && prec == PPCA_PREC_ACCURATE);
    const int64_t b = h->params.batch;
    return tc && b <= h->x.n && xpass_tc_row0_same(h->x, b, prec, h->sched, h->num_sms);
}

ppca_status build_step_graph(ppca_handle* h, const StepGraphKey& key) {
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    if (!h->gstream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
    }
    const int m = h->m;
    const int64_t n = h->x.n, d = h->x.d, b = h->params.batch, per_epoch = (n + b - 1) / b;
    const bool oja = h->method == PPCA_OJA;
    cudaStream_t st = h->gstream;
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kStepGraph && e == cudaSuccess; ++i) {
        e = primer_step_begin(h->pstep, per_epoch, b, oja ? h->params.lr : 0.0, oja ? h->params.lr_offset : 1.0, st);
        if (e == cudaSuccess)
            e = xpass_tc(h->x, h->V, m, 0, b, h->Z, prime_prec(h), h->tc, h->sched, h->status, h->num_sms, st,
                         &h->pstep->row0);
        if (e == cudaSuccess) e = gram_df(h->V, h->Z, d, m, h->G, h->gram_part, st);
        if (e == cudaSuccess)
            e = oja ? oja_update(h->V, h->Z, h->G, d, m, 0.0, st, &h->pstep->c)
                    : eigengame_update(h->V, h->buf, h->Z, h->G, d, m, 1.0 / (double)b, h->params.lr,
                                       h->params.momentum, h->eg, st);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->gexec = nullptr;
        return fail(PPCA_ERR_CUDA, "capturing the minibatch steps failed: %s", cudaGetErrorString(e));
    }
    static_assert(sizeof(StepGraphKey) <= sizeof(h->gkey), "step graph key");
    std::memcpy(h->gkey, &key, sizeof key);
    return PPCA_OK;
}

// Runs as many whole graphs of full-minibatch steps as fit in `remaining` from
// step h->t on (none if the next kStepGraph steps hold the epoch's partial
// batch); *done = the steps run.
ppca_status step_graphs(ppca_handle* h, int64_t remaining, int64_t* done) {
    *done = 0;
    if (remaining < kStepGraph || !step_graph_eligible(h)) return PPCA_OK;
    const int64_t n = h->x.n, b = h->params.batch, per_epoch = (n + b - 1) / b;
    const int64_t full = n % b == 0 ? per_epoch : per_epoch - 1;     // full batches per epoch
    int64_t blocks = 0;
    for (int64_t t = h->t; remaining - blocks * kStepGraph >= kStepGraph; t += kStepGraph) {
        if (n % b != 0 && (t % per_epoch) + kStepGraph > full) break;
        ++blocks;
    }
    if (blocks == 0) return PPCA_OK;
    StepGraphKey key;
    std::memset(&key, 0, sizeof key);
    key.method = h->method;
    key.m = h->m;
    key.dtype = h->x.dtype;
    key.prec = prime_prec(h);
    key.n = n;
    key.d = h->x.d;
    key.ld = h->x.ld;
    key.batch = b;
    key.x = h->x.ptr;
    key.ws = h->ws;
    key.lr = h->params.lr;
    key.lr_offset = h->params.lr_offset;
    key.momentum = h->params.momentum;
    key.sched = h->sched;
    if (!h->gexec || std::memcmp(h->gkey, &key, sizeof key) != 0) PPCA_TRY(build_step_graph(h, key));
    CUDA_TRY(cudaEventRecord(h->gev_in, h->stream));
    CUDA_TRY(cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
    CUDA_TRY(primer_step_set(h->pstep, h->t, h->gstream));
    for (int64_t i = 0; i < blocks; ++i) CUDA_TRY(cudaGraphLaunch(h->gexec, h->gstream));
    CUDA_TRY(cudaEventRecord(h->gev_out, h->gstream));
    CUDA_TRY(cudaStreamWaitEvent(h->stream, h->gev_out, 0));
    h->t += blocks * kStepGraph;
    *done = blocks * kStepGraph;
    return PPCA_OK;
}

ppca_status run_steps(ppca_handle* h, int64_t T) {
    const int m = h->m;
    const int64_t n = h->x.n, d = h->x.d;
    if (h->method == PPCA_POWER_SEQ) return run_power_seq(h, T);
    if (h->method == PPCA_OJA || h->method == PPCA_EIGENGAME) {
        int64_t i = 0;
        while (i < T) {
            int64_t g = 0;
            PPCA_TRY(step_graphs(h, T - i, &g));
            i += g;
            if (i < T) {
                PPCA_TRY(minibatch_step(h));
                ++i;
            }
        }
        return PPCA_OK;
    }
    for (int64_t i = 0; i < T; ++i) {
        switch (h->method) {
        case PPCA_POWER:
            PPCA_TRY(run_xpass(h, h->x, h->V, m, 0, n, h->Z, prime_prec(h)));
            PPCA_TRY(allreduce(h, h->Z, d * m, 4));                               // Z over all ranks' rows
            PPCA_TRY(run_orth(h, h->Z, h->V, m, /*span_only=*/true));
            ++h->iters;
            break;
        default:
            return fail(PPCA_ERR_STATE, "no priming method set");
        }
    }
    return PPCA_OK;
}

constexpr uint32_t kStateMagic = 0x50504341u;   // "PPCA"

struct StateHeader {
    uint32_t magic;
    int32_t version;
    int64_t n, d;
    int32_t method, m;
    int64_t t, iters;
    ppca_prime_params params;
};

}  // namespace

// ============================================================================ C ABI

extern "C" {

int32_t ppca_version(void) { return (1 << 16) | 0; }

const char* ppca_last_error(void) { return g_last_error.c_str(); }

ppca_status ppca_prime_params_default(ppca_prime_params* p, ppca_method method) {
    if (!p) return fail(PPCA_ERR_INVALID, "params is NULL");
    std::memset(p, 0, sizeof *p);
    switch (method) {
    case PPCA_POWER:
        break;
    case PPCA_OJA:
        p->batch = 256;
        p->lr = 1.0;
        p->lr_offset = 100.0;
        break;
    case PPCA_EIGENGAME:
        p->batch = 1024;
        p->lr = 0.05;
        p->momentum = 0.9;
        break;
    case PPCA_POWER_SEQ:
        p->eps = 1e-6;
        break;
    default:
        return fail(PPCA_ERR_INVALID, "unknown method %d", (int)method);
    }
    return PPCA_OK;
}

ppca_status ppca_create(ppca_handle** out, const void* X, int64_t n, int64_t d, int64_t ld, ppca_dtype dtype,
                        const float* row_scales, void* stream) {
    if (!out) return fail(PPCA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    PPCA_TRY(validate_x(X, n, d, ld, dtype, row_scales));
    ppca_handle* h = new (std::nothrow) ppca_handle();
    if (!h) return fail(PPCA_ERR_OOM, "host allocation failed");
    h->x.ptr = X;
    h->x.n = n;
    h->x.d = d;
    h->x.ld = ld;
    h->x.dtype = dtype;
    h->x.scales = row_scales;
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->status), 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, 256, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->status) cudaFree(h->status);
        delete h;
        return fail(PPCA_ERR_CUDA, "device setup failed: %s", cudaGetErrorString(e));
    }
    *out = h;
    return PPCA_OK;
}

ppca_status ppca_set_refine(ppca_handle* h, const void* X_refine, int64_t ld, ppca_dtype dtype) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (!X_refine) {
        h->has_ref = false;
        return PPCA_OK;
    }
    if (dtype == PPCA_FP8_E4M3) return fail(PPCA_ERR_INVALID, "the refine copy must be FP32 or BF16");
    PPCA_TRY(validate_x(X_refine, h->x.n, h->x.d, ld, dtype, nullptr));
    h->xref = h->x;
    h->xref.ptr = X_refine;
    h->xref.ld = ld;
    h->xref.dtype = dtype;
    h->xref.scales = nullptr;
    h->has_ref = true;
    return PPCA_OK;
}

ppca_status ppca_set_workspace_limit(ppca_handle* h, int64_t bytes) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (bytes < 0) return fail(PPCA_ERR_INVALID, "negative limit");
    h->ws_limit = bytes;
    return PPCA_OK;
}

static ppca_status check_m(const ppca_handle* h, int32_t m) {
    const int64_t cap = std::min<int64_t>(std::min<int64_t>(h->x.d, h->x.n - 1), kMaxM);
    if (m < 1 || m > cap)
        return fail(PPCA_ERR_INVALID, "m = k + l = %d out of range [1, min(d, n-1, %d) = %lld]", m, kMaxM,
                    (long long)cap);
    return PPCA_OK;
}

ppca_status ppca_prime(ppca_handle* h, ppca_method method, int32_t m, int64_t T, const ppca_prime_params* p) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (method != PPCA_POWER && method != PPCA_OJA && method != PPCA_EIGENGAME && method != PPCA_POWER_SEQ)
        return fail(PPCA_ERR_INVALID, "unknown method %d", (int)method);
    PPCA_TRY(check_m(h, m));
    if (T < 0) return fail(PPCA_ERR_INVALID, "T = %lld < 0", (long long)T);
    ppca_prime_params prm;
    if (p) {
        prm = *p;
    } else {
        PPCA_TRY(ppca_prime_params_default(&prm, method));
    }
    if (prm.reserved != 0) return fail(PPCA_ERR_INVALID, "reserved field must be 0");
    if (prm.precision < PPCA_PREC_AUTO || prm.precision > PPCA_PREC_ACCURATE)
        return fail(PPCA_ERR_INVALID, "unknown precision %d", prm.precision);
    if (method == PPCA_POWER_SEQ && !(prm.eps >= 0.0)) return fail(PPCA_ERR_INVALID, "eps must be >= 0");
    if (method == PPCA_OJA || method == PPCA_EIGENGAME) {
        if (prm.batch <= 0) return fail(PPCA_ERR_INVALID, "batch = %lld must be > 0", (long long)prm.batch);
        if (!(prm.lr > 0.0)) return fail(PPCA_ERR_INVALID, "lr must be > 0");
        if (method == PPCA_OJA && !(prm.lr_offset + (double)prm.t0 > 0.0))
            return fail(PPCA_ERR_INVALID, "lr_offset + t0 must be > 0");
        if (prm.t0 < 0) return fail(PPCA_ERR_INVALID, "t0 < 0");
    }
    PPCA_TRY(ensure_workspace(h, m));
    h->method = method;
    h->m = m;
    h->params = prm;
    h->t = prm.t0;
    h->iters = 0;
    const int64_t d = h->x.d;
    if (prm.V0) {
        CUDA_TRY(cudaMemcpyAsync(h->V, prm.V0, (size_t)d * m * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    } else {
        CUDA_TRY(init_gaussian(h->V, d, m, prm.seed, h->stream));
    }
    CUDA_TRY(cudaMemsetAsync(h->buf, 0, (size_t)d * m * sizeof(float), h->stream));
    PPCA_TRY(run_orth(h, h->V, h->V, m));
    h->params.V0 = nullptr;   // not retained
    return run_steps(h, T);
}

ppca_status ppca_prime_continue(ppca_handle* h, int64_t T) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (h->method < 0) return fail(PPCA_ERR_STATE, "ppca_prime was not called");
    if (h->method == PPCA_POWER_SEQ)
        return fail(PPCA_ERR_UNSUPPORTED, "the sequential power method runs each direction to completion");
    if (T < 0) return fail(PPCA_ERR_INVALID, "T < 0");
    return run_steps(h, T);
}

ppca_status ppca_finalize(ppca_handle* h, int32_t k, float* E, double* lambda, ppca_precision precision) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (h->method < 0) return fail(PPCA_ERR_STATE, "finalize before prime");
    const int m = h->m;
    if (k < 1 || k > m) return fail(PPCA_ERR_INVALID, "k = %d out of range [1, m = %d]", k, m);
    if (!E || !lambda) return fail(PPCA_ERR_INVALID, "E or lambda is NULL");
    if (precision < PPCA_PREC_AUTO || precision > PPCA_PREC_ACCURATE)
        return fail(PPCA_ERR_INVALID, "unknown precision %d", (int)precision);
    const ppca_precision prec = precision == PPCA_PREC_AUTO ? PPCA_PREC_ACCURATE : precision;
    const int64_t d = h->x.d, n = h->x.n;
    PPCA_TRY(run_orth(h, h->V, h->Q, m));                                          // step 2: span
    const XView& xf = h->has_ref ? h->xref : h->x;
    PPCA_TRY(run_gram(h, xf, h->Q, m, 0, n, h->G, prec));                          // step 3: G = (XQ)^T XQ
    PPCA_TRY(allreduce(h, h->G, (int64_t)m * m, 8));                               // over all ranks' rows
    CUDA_TRY(eigh_small(h->G, m, h->w, h->U, h->jac, h->status, h->stream));       // step 4: full-PCA
    CUDA_TRY(rotate_and_sign(h->Q, d, m, h->U, h->w, k, 1.0 / (double)rows_total(h), E, lambda,
                             h->stream));                                          // step 5
    return PPCA_OK;
}

ppca_status ppca_get_basis(const ppca_handle* h, float* V_out) {
    if (!h || !V_out) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (h->method < 0) return fail(PPCA_ERR_STATE, "no primed basis");
    CUDA_TRY(cudaMemcpyAsync(V_out, h->V, (size_t)h->x.d * h->m * sizeof(float), cudaMemcpyDeviceToDevice,
                             h->stream));
    return PPCA_OK;
}

ppca_status ppca_upload(ppca_handle* h, const void* X_host, int64_t ld_host, const float* row_scales_host) {
    if (!h || !X_host) return fail(PPCA_ERR_INVALID, "NULL argument");
    const XView& x = h->x;
    if (ld_host < x.d) return fail(PPCA_ERR_INVALID, "ld_host = %lld < d = %lld", (long long)ld_host, (long long)x.d);
    if ((x.dtype == PPCA_FP8_E4M3) != (row_scales_host != nullptr))
        return fail(PPCA_ERR_INVALID, "row_scales_host must be given for FP8 data and only for FP8 data");
    const size_t esz = (size_t)dtype_size(x.dtype);
    void* dst = const_cast<void*>(x.ptr);     // the caller's device buffer, written on request
    if (ld_host == x.ld && x.ld == x.d)
        CUDA_TRY(cudaMemcpyAsync(dst, X_host, (size_t)x.n * x.d * esz, cudaMemcpyHostToDevice, h->stream));
    else
        CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)x.ld * esz, X_host, (size_t)ld_host * esz, (size_t)x.d * esz,
                                   (size_t)x.n, cudaMemcpyHostToDevice, h->stream));
    if (row_scales_host)
        CUDA_TRY(cudaMemcpyAsync(const_cast<float*>(x.scales), row_scales_host, (size_t)x.n * sizeof(float),
                                 cudaMemcpyHostToDevice, h->stream));
    return PPCA_OK;
}

ppca_status ppca_finalize_sampled(ppca_handle* h, int32_t k, float* E, double* lambda, ppca_precision precision,
                                  double fraction, uint64_t seed, int64_t* rows_used) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (h->method < 0) return fail(PPCA_ERR_STATE, "finalize before prime");
    const int m = h->m;
    if (k < 1 || k > m) return fail(PPCA_ERR_INVALID, "k = %d out of range [1, m = %d]", k, m);
    if (!E || !lambda) return fail(PPCA_ERR_INVALID, "E or lambda is NULL");
    if (precision < PPCA_PREC_AUTO || precision > PPCA_PREC_ACCURATE)
        return fail(PPCA_ERR_INVALID, "unknown precision %d", (int)precision);
    if (!(fraction > 0.0 && fraction <= 1.0)) return fail(PPCA_ERR_INVALID, "fraction must be in (0, 1]");
    const XView& xf = h->has_ref ? h->xref : h->x;
    if (!tc_pass_supported(xf, m) || xf.dtype == PPCA_FP8_E4M3 || h->sched.engine == 2)
        return fail(PPCA_ERR_UNSUPPORTED, "the sampled pPCA step runs on tensor cores over BF16 or FP32 data");
    const ppca_precision prec = precision == PPCA_PREC_AUTO ? PPCA_PREC_ACCURATE : precision;
    const int64_t d = h->x.d, n = xf.n, nt = (n + 127) / 128;
    // the kept blocks (the device kernel builds the same list from the same rule)
    int64_t nsel = 0, rows = 0, best_t = 0;
    uint64_t best_u = ~0ull;
    for (int64_t t = 0; t < nt; ++t) {
        const uint64_t u = sample_block_u(seed, t);
        if (u < best_u) {
            best_u = u;
            best_t = t;
        }
        if (sample_block_kept(u, fraction)) {
            ++nsel;
            rows += std::min<int64_t>(128, n - t * 128);
        }
    }
    int64_t forced = -1;
    if (nsel == 0) {
        forced = best_t;
        nsel = 1;
        rows = std::min<int64_t>(128, n - best_t * 128);
    }
    CUDA_TRY(sample_blocks(n, fraction, seed, forced, h->tile_rows, h->stream));
    PPCA_TRY(run_orth(h, h->V, h->Q, m));                                          // step 2: span
    cudaEvent_t ev_end = nullptr;
    PPCA_TRY(pass_timer(h, prec, rows, &ev_end));
    CUDA_TRY(projected_gram_tc_blocks(xf, h->Q, m, h->tile_rows, (int)nsel, h->G, prec, h->sched.flush, h->tc,
                                      h->status, h->num_sms, h->stream));         // step 3 on the sample
    if (ev_end) CUDA_TRY(cudaEventRecord(ev_end, h->stream));
    PPCA_TRY(allreduce(h, h->G, (int64_t)m * m, 8));                               // each rank's sample
    PPCA_TRY(global_rows(h, rows, &rows));
    CUDA_TRY(eigh_small(h->G, m, h->w, h->U, h->jac, h->status, h->stream));       // step 4
    CUDA_TRY(rotate_and_sign(h->Q, d, m, h->U, h->w, k, 1.0 / (double)rows, E, lambda, h->stream));
    if (rows_used) *rows_used = rows;
    return PPCA_OK;
}

ppca_status ppca_variance_captured(ppca_handle* h, const float* E, int32_t k, double* var, ppca_precision precision) {
    if (!h || !E || !var) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (k < 1 || k > kMaxM || k > h->x.d) return fail(PPCA_ERR_INVALID, "k = %d out of range", k);
    if (precision < PPCA_PREC_AUTO || precision > PPCA_PREC_ACCURATE)
        return fail(PPCA_ERR_INVALID, "unknown precision %d", (int)precision);
    const ppca_precision prec = precision == PPCA_PREC_AUTO ? PPCA_PREC_ACCURATE : precision;
    if (h->method >= 0 && k > h->ws_m)      // a larger workspace would drop the primed basis
        return fail(PPCA_ERR_INVALID, "k = %d exceeds the primed width m = %d", k, h->ws_m);
    PPCA_TRY(ensure_workspace(h, std::max(k, h->ws_m)));
    const XView& xf = h->has_ref ? h->xref : h->x;
    PPCA_TRY(run_gram(h, xf, E, k, 0, xf.n, h->G, prec));                         // G = (X E)^T (X E)
    PPCA_TRY(allreduce(h, h->G, (int64_t)k * k, 8));                               // over all ranks' rows
    CUDA_TRY(cudaMemcpy2DAsync(var, sizeof(double), h->G, (size_t)(k + 1) * sizeof(double), sizeof(double), (size_t)k,
                               cudaMemcpyDeviceToDevice, h->stream));              // its diagonal
    return PPCA_OK;
}

ppca_status ppca_finalize_host(ppca_handle* h, int32_t k, float* E_host, double* lambda_host,
                               ppca_precision precision) {
    if (!h || !E_host || !lambda_host) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (h->method < 0) return fail(PPCA_ERR_STATE, "finalize before prime");
    PPCA_TRY(ppca_finalize(h, k, h->E_res, h->lam_res, precision));
    CUDA_TRY(cudaMemcpyAsync(E_host, h->E_res, (size_t)k * h->x.d * sizeof(float), cudaMemcpyDeviceToHost,
                             h->stream));
    CUDA_TRY(cudaMemcpyAsync(lambda_host, h->lam_res, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    return PPCA_OK;
}

ppca_status ppca_sync(ppca_handle* h) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return check_status_word(h->status);
}

}  // extern "C"

// The device status word after the work that writes it has finished: an error
// code is reported (and the word cleared for the next call).
ppca_status check_status_word(int* status) {
    int st = 0;
    CUDA_TRY(cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != kDevOk) {
        CUDA_TRY(cudaMemset(status, 0, sizeof(int)));
        switch (st) {
        case kDevCholeskyBreakdown:
            return fail(PPCA_ERR_NUMERICAL, "CholeskyQR2: non-positive pivot (basis numerically rank-deficient)");
        case kDevJacobiNoConverge:
            return fail(PPCA_ERR_NUMERICAL, "Jacobi eigensolver did not converge within its sweep cap");
        case kDevWaitTimeout:
            return fail(PPCA_ERR_TIMEOUT, "a bounded device-side wait ran out");
        default:
            return fail(PPCA_ERR_NUMERICAL, "device status %d", st);
        }
    }
    return PPCA_OK;
}

extern "C" {

ppca_status ppca_get_state(ppca_handle* h, void* buf, int64_t* bytes) {
    if (!h || !bytes) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (h->method < 0) return fail(PPCA_ERR_STATE, "no priming state");
    const size_t dm = (size_t)h->x.d * h->m * sizeof(float);
    const int64_t need = (int64_t)(sizeof(StateHeader) + 2 * dm);
    if (!buf) {
        *bytes = need;
        return PPCA_OK;
    }
    if (*bytes < need) return fail(PPCA_ERR_INVALID, "state buffer too small (%lld < %lld)", (long long)*bytes,
                                   (long long)need);
    StateHeader hd{};
    hd.magic = kStateMagic;
    hd.version = 2;                  // 2: the prime parameters carry eps
    hd.n = h->x.n;
    hd.d = h->x.d;
    hd.method = h->method;
    hd.m = h->m;
    hd.t = h->t;
    hd.iters = h->iters;
    hd.params = h->params;
    hd.params.V0 = nullptr;
    std::memcpy(buf, &hd, sizeof hd);
    char* p = static_cast<char*>(buf) + sizeof hd;
    CUDA_TRY(cudaMemcpyAsync(p, h->V, dm, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(p + dm, h->buf, dm, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    *bytes = need;
    return PPCA_OK;
}

ppca_status ppca_set_state(ppca_handle* h, const void* buf, int64_t bytes) {
    if (!h || !buf) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (bytes < (int64_t)sizeof(StateHeader)) return fail(PPCA_ERR_INVALID, "state buffer too small");
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kStateMagic || hd.version != 2) return fail(PPCA_ERR_INVALID, "not a ppca state buffer");
    if (hd.n != h->x.n || hd.d != h->x.d) return fail(PPCA_ERR_INVALID, "state is for another (n, d)");
    PPCA_TRY(check_m(h, hd.m));
    const size_t dm = (size_t)h->x.d * hd.m * sizeof(float);
    if (bytes < (int64_t)(sizeof hd + 2 * dm)) return fail(PPCA_ERR_INVALID, "state buffer truncated");
    PPCA_TRY(ensure_workspace(h, hd.m));
    h->method = hd.method;
    h->m = hd.m;
    h->t = hd.t;
    h->iters = hd.iters;
    h->params = hd.params;
    const char* p = static_cast<const char*>(buf) + sizeof hd;
    CUDA_TRY(cudaMemcpyAsync(h->V, p, dm, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->buf, p + dm, dm, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return PPCA_OK;
}

ppca_status ppca_set_schedule(ppca_handle* h, const ppca_schedule* s) {
    if (!h || !s) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (s->fused < -1 || s->fused > 1 || s->producers < 0 || s->window < 0 || s->flush < 0 || s->engine < 0 ||
        s->engine > 2 || s->kparts < 0 || s->kparts > 2 || s->l2_keep < 0 || s->l2_keep > 100 || s->fp8_mma < 0 ||
        s->fp8_mma > 2)
        return fail(PPCA_ERR_INVALID, "schedule out of range");
    h->sched.fused = s->fused;
    h->sched.producers = s->producers;
    h->sched.window = s->window;
    h->sched.flush = s->flush;
    h->sched.engine = s->engine;
    h->sched.kparts = s->kparts;
    h->sched.l2_keep = s->l2_keep;
    h->sched.fp8_mma = s->fp8_mma == 2 ? 0 : 1;
    return PPCA_OK;
}

ppca_status ppca_set_allreduce(ppca_handle* h, ppca_allreduce_fn fn, void* ctx, int64_t n_total, void* staging,
                               int64_t staging_bytes) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    if (!fn) {
        h->ar_fn = nullptr;
        h->ar_ctx = h->ar_stage = nullptr;
        h->ar_stage_bytes = h->n_total = 0;
        return PPCA_OK;
    }
    if (n_total < h->x.n) return fail(PPCA_ERR_INVALID, "n_total = %lld < the local rows %lld", (long long)n_total,
                                      (long long)h->x.n);
    if ((staging == nullptr) != (staging_bytes == 0) || staging_bytes < 0)
        return fail(PPCA_ERR_INVALID, "staging buffer and its size must be given together");
    h->ar_fn = fn;
    h->ar_ctx = ctx;
    h->ar_stage = staging;
    h->ar_stage_bytes = staging_bytes;
    h->n_total = n_total;
    return PPCA_OK;
}

ppca_status ppca_set_wait_limit(uint64_t ns) {
    if (ns > 60ull * 1000000000ull) return fail(PPCA_ERR_INVALID, "wait limit %llu ns above 60 s", (unsigned long long)ns);
    CUDA_TRY(pass_tc_set_wait_limit(ns));
    CUDA_TRY(pass_gram_set_wait_limit(ns));
    return PPCA_OK;
}

namespace {

ppca_schedule to_abi(const TcSchedule& t) {
    ppca_schedule s{};
    s.fused = t.fused;
    s.producers = t.producers;
    s.window = t.window;
    s.flush = t.flush;
    s.engine = t.engine;
    s.kparts = t.kparts;
    s.l2_keep = t.l2_keep;
    s.fp8_mma = t.fp8_mma == 0 ? 2 : 1;
    return s;
}

// Time the fast pass under each candidate schedule; keep the fastest on the handle.
ppca_status autotune_handle(ppca_handle* h, int m, int64_t rows, int reps, bool allow_fused, TcSchedule* out) {
    PPCA_TRY(ensure_workspace(h, std::max(m, h->ws_m)));
    const XView& x = h->x;
    if (rows <= 0 || rows > x.n) rows = x.n;
    std::vector<TcSchedule> cands;
    TcSchedule base = h->sched;
    if (tc_pass_supported(x, m)) {
        TcSchedule c = base;
        c.engine = 1;
        c.fused = 0;
        cands.push_back(c);
        if (allow_fused && x.dtype == PPCA_BF16) {
            c.fused = 1;
            for (int kp = 2; kp >= 1; --kp) {           // half-K or whole-K producer tiles
                c.kparts = kp;
                cands.push_back(c);
            }
            c.l2_keep = 100;                            // every tile protected in L2
            cands.push_back(c);
            c.l2_keep = base.l2_keep;
        }
    }
    {
        TcSchedule c = base;
        c.engine = 2;
        c.fused = 0;
        cands.push_back(c);
    }
    CUDA_TRY(init_gaussian(h->Q, x.d, m, 0x5eedull, h->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = -1.f;
    TcSchedule best = cands.front();
    ppca_status st = PPCA_OK;
    for (const TcSchedule& c : cands) {
        h->sched = c;
        st = run_xpass(h, x, h->Q, m, 0, rows, h->T, PPCA_PREC_FAST);     // warm-up
        if (st != PPCA_OK) break;
        float ms_min = -1.f;
        for (int r = 0; r < std::max(reps, 1) && st == PPCA_OK; ++r) {
            cudaEventRecord(e0, h->stream);
            st = run_xpass(h, x, h->Q, m, 0, rows, h->T, PPCA_PREC_FAST);
            cudaEventRecord(e1, h->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = fail(PPCA_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms_min < 0.f || ms < ms_min) ms_min = ms;
        }
        if (st != PPCA_OK) break;
        if (best_ms < 0.f || ms_min < best_ms) {
            best_ms = ms_min;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->sched = st == PPCA_OK ? best : base;
    if (st != PPCA_OK) return st;
    if (out) *out = best;
    return PPCA_OK;
}

}  // namespace

ppca_status ppca_autotune(ppca_handle* h, int32_t m, int64_t rows, int32_t reps, ppca_schedule* best) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    PPCA_TRY(check_m(h, m));
    if (rows < 0) return fail(PPCA_ERR_INVALID, "rows < 0");
    TcSchedule t;
    PPCA_TRY(autotune_handle(h, m, rows, reps, true, &t));
    if (best) *best = to_abi(t);
    return PPCA_OK;
}

ppca_status ppca_set_timing(ppca_handle* h, int32_t enable) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    h->timing = enable != 0;
    h->events_used = 0;
    for (int i = 0; i < 3; ++i) {
        h->timed_passes[i] = 0;
        h->timed_rows[i] = 0;
    }
    h->launch_base = launches_so_far();
    return PPCA_OK;
}

ppca_status ppca_get_timing(ppca_handle* h, ppca_timing* out) {
    if (!h || !out) return fail(PPCA_ERR_INVALID, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    double ms[3] = {0.0, 0.0, 0.0};
    for (size_t i = 0; i < h->events_used; ++i) {
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, h->events[i].first, h->events[i].second));
        ms[h->event_prec[i]] += e;
    }
    for (int i = 0; i < 3; ++i) {
        out->pass_ms[i] = ms[i];
        out->passes[i] = h->timed_passes[i];
        out->pass_rows[i] = h->timed_rows[i];
    }
    out->launches = launches_so_far() - h->launch_base;
    return PPCA_OK;
}

ppca_status ppca_destroy(ppca_handle* h) {
    if (!h) return PPCA_OK;
    cudaStreamSynchronize(h->stream);
    for (auto& pr : h->events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gstream) {
        cudaStreamSynchronize(h->gstream);
        cudaStreamDestroy(h->gstream);
    }
    if (h->gev_in) cudaEventDestroy(h->gev_in);
    if (h->gev_out) cudaEventDestroy(h->gev_out);
    if (h->ws) cudaFree(h->ws);
    if (h->status) cudaFree(h->status);
    delete h;
    return PPCA_OK;
}

ppca_status ppca_set_step_graphs(ppca_handle* h, int32_t enable) {
    if (!h) return fail(PPCA_ERR_INVALID, "handle is NULL");
    h->step_graphs = enable != 0;
    return PPCA_OK;
}

ppca_status ppca_xpass(ppca_handle* h, const float* V, int32_t m, int64_t r0, int64_t r1, float* Z,
                       ppca_precision precision) {
    if (!h || !V || !Z) return fail(PPCA_ERR_INVALID, "NULL argument");
    PPCA_TRY(check_m(h, m));
    if (r0 < 0 || r1 > h->x.n || r0 >= r1)
        return fail(PPCA_ERR_INVALID, "row range [%lld, %lld) invalid for n = %lld", (long long)r0, (long long)r1,
                    (long long)h->x.n);
    if (precision < PPCA_PREC_AUTO || precision > PPCA_PREC_ACCURATE)
        return fail(PPCA_ERR_INVALID, "unknown precision %d", (int)precision);
    PPCA_TRY(ensure_workspace(h, std::max(m, h->ws_m)));
    const ppca_precision prec = precision == PPCA_PREC_AUTO ? PPCA_PREC_FAST : precision;
    return run_xpass(h, h->x, V, m, r0, r1, Z, prec);
}

ppca_status ppca_projected_gram(ppca_handle* h, const float* Q, int32_t m, int64_t r0, int64_t r1, double* G,
                                ppca_precision precision) {
    if (!h || !Q || !G) return fail(PPCA_ERR_INVALID, "NULL argument");
    PPCA_TRY(check_m(h, m));
    if (r0 < 0 || r1 > h->x.n || r0 >= r1)
        return fail(PPCA_ERR_INVALID, "row range [%lld, %lld) invalid for n = %lld", (long long)r0, (long long)r1,
                    (long long)h->x.n);
    if (precision < PPCA_PREC_AUTO || precision > PPCA_PREC_ACCURATE)
        return fail(PPCA_ERR_INVALID, "unknown precision %d", (int)precision);
    PPCA_TRY(ensure_workspace(h, std::max(m, h->ws_m)));
    const ppca_precision prec = precision == PPCA_PREC_AUTO ? PPCA_PREC_ACCURATE : precision;
    return run_gram(h, h->has_ref ? h->xref : h->x, Q, m, r0, r1, G, prec);
}

ppca_status ppca_orthonormalize(ppca_handle* h, const float* V, float* Q, int32_t m) {
    if (!h || !V || !Q) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (m < 1 || m > kMaxM || m > h->x.d) return fail(PPCA_ERR_INVALID, "m = %d out of range", m);
    PPCA_TRY(ensure_workspace(h, std::max(m, h->ws_m)));
    return run_orth(h, V, Q, m);
}

ppca_status ppca_eigh(ppca_handle* h, const double* G, int32_t m, double* w, double* U) {
    if (!h || !G || !w || !U) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (m < 1 || m > kMaxM) return fail(PPCA_ERR_INVALID, "m = %d out of range [1, %d]", m, kMaxM);
    PPCA_TRY(ensure_workspace(h, std::max(m, h->ws_m)));
    CUDA_TRY(eigh_small(G, m, w, U, h->jac, h->status, h->stream));
    return PPCA_OK;
}

ppca_status ppca_eigh_noalloc(const double* G, int32_t m, double* w, double* U, int* status, void* stream) {
    if (!G || !w || !U) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (m < 1 || m > kMaxM)
        return fail(PPCA_ERR_INVALID, "m = %d out of range [1, %d]: the fixed %zu-byte scratch holds m <= %d", m,
                    kMaxM, eigh_noalloc_scratch_bytes(), kMaxM);
    CUDA_TRY(eigh_small_noalloc(G, m, w, U, status, static_cast<cudaStream_t>(stream)));
    return PPCA_OK;
}

ppca_status ppca_quantize_bf16(const float* X, int64_t n, int64_t d, int64_t ld_in, uint16_t* out, int64_t ld_out,
                               void* stream) {
    if (!X || !out) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (n < 0 || d < 0 || ld_in < d || ld_out < d) return fail(PPCA_ERR_INVALID, "bad shape");
    CUDA_TRY(quantize_bf16(X, n, d, ld_in, out, ld_out, static_cast<cudaStream_t>(stream)));
    return PPCA_OK;
}

ppca_status ppca_quantize_fp8(const float* X, int64_t n, int64_t d, int64_t ld_in, uint8_t* out, int64_t ld_out,
                              float* scales, void* stream) {
    if (!X || !out || !scales) return fail(PPCA_ERR_INVALID, "NULL argument");
    if (n < 0 || d < 0 || ld_in < d || ld_out < d) return fail(PPCA_ERR_INVALID, "bad shape");
    CUDA_TRY(quantize_fp8(X, n, d, ld_in, out, ld_out, scales, static_cast<cudaStream_t>(stream)));
    return PPCA_OK;
}

}  // extern "C"

// ============================================================================ batches

struct ppca_batch {
    std::vector<ppca_instance_desc> descs;
    cudaStream_t user_stream = nullptr;   // the caller's stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;        // the batch's own stream: captured, and where the graph runs
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<ppca_handle*> slots;
    std::vector<cudaStream_t> slot_streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;                  // kernel launches captured in the graph
    std::vector<TcSchedule> inst_sched;   // per instance, after ppca_batch_autotune
    bool prime_bf16 = false;              // FP32 instances primed on a BF16 rounding of X
    std::vector<void*> prime_buf;         // per slot: that rounding, for its largest FP32 instance

    // Lockstep: every instance's power iterations and pPCA step in grouped
    // launches (grouped.h), one launch per kernel kind and iteration for the
    // whole batch; the slots are not used.
    bool lockstep = true;                 // allowed (ppca_batch_set_lockstep)
    bool grouped = false;                 // the captured graph primes in lockstep
    void* g_mem = nullptr;                // per-instance buffers, tables, descriptors
    GInst* g_inst = nullptr;              // device: one per instance
    GMaps* g_maps = nullptr;              // device: one per instance
    int* g_status = nullptr;              // device status word of the lockstep kernels
    std::vector<GInst> g_host;
    GTable t_quant{}, t_splitq{}, t_xv{}, t_xty{}, t_dm{}, t_gram{}, t_reduce{}, t_apply{};
    GTable t_ygen32{}, t_ygen16{}, t_ychunks{}, t_gred{}, t_rayleigh{}, t_rotate{}, t_sign{};
    bool any_vout = false;
    const float* const* g_x32 = nullptr;  // device: FP32 X of each instance (quantize)
    const int64_t* g_ld32 = nullptr;
    bool any_f32 = false;
    int g_max_m = 0;
    int num_sms = 0;
    cudaEvent_t g_done = nullptr;
};

namespace {

void free_slot(ppca_handle* h) {
    if (!h) return;
    if (h->ws) cudaFree(h->ws);
    if (h->status) cudaFree(h->status);
    delete h;
}

void free_batch(ppca_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto* h : b->slots) free_slot(h);
    for (auto p : b->prime_buf) cudaFree(p);
    if (b->g_mem) cudaFree(b->g_mem);
    if (b->g_status) cudaFree(b->g_status);
    if (b->g_done) cudaEventDestroy(b->g_done);
    for (auto s : b->slot_streams) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

XView view_of(const ppca_instance_desc& ds) {
    XView x;
    x.ptr = ds.X;
    x.n = ds.n;
    x.d = ds.d;
    x.ld = ds.ld;
    x.dtype = (ppca_dtype)ds.dtype;
    x.scales = ds.row_scales;
    return x;
}

inline int64_t bf16_ld(int64_t d) { return (d + 7) / 8 * 8; }    // 16-byte row pitch

// Point slot h at instance i: its priming data is X itself, or (BF16 priming of FP32
// data) the BF16 rounding of X enqueued now into the slot's buffer, with X as the
// pPCA step's refine copy.
ppca_status bind_instance(ppca_batch* b, ppca_handle* h, int slot, const ppca_instance_desc& ds) {
    h->x = view_of(ds);
    h->has_ref = false;
    if (!b->prime_bf16 || ds.dtype != PPCA_F32) return PPCA_OK;
    const int64_t ldb = bf16_ld(ds.d);
    CUDA_TRY(quantize_bf16(static_cast<const float*>(ds.X), ds.n, ds.d, ds.ld,
                           static_cast<uint16_t*>(b->prime_buf[slot]), ldb, h->stream));
    h->xref = h->x;
    h->has_ref = true;
    h->x.ptr = b->prime_buf[slot];
    h->x.ld = ldb;
    h->x.dtype = PPCA_BF16;
    return PPCA_OK;
}

// ---- lockstep batch

inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// A lockstep batch: all instances prime on BF16 data (BF16 X, or FP32 X with
// BF16 priming and d % 8 == 0), with one T for all, on the tensor-core pass.
bool lockstep_eligible(const ppca_batch* b) {
    if (!b->lockstep) return false;
    const int T = b->descs[0].T;
    for (const auto& ds : b->descs) {
        if (ds.T != T) return false;
        const bool bf16 = ds.dtype == PPCA_BF16;
        const bool f32 = ds.dtype == PPCA_F32 && b->prime_bf16 && ds.d % 8 == 0;
        if (!bf16 && !f32) return false;
        XView x = view_of(ds);
        x.dtype = PPCA_BF16;
        if (!tc_pass_supported(x, ds.m)) return false;
    }
    return true;
}

// Buffers, work tables and TMA descriptors of the lockstep batch (once, before
// the capture).  Returns false, with nothing allocated, when the device memory
// is not there (the batch then primes on its slots).
bool prepare_lockstep(ppca_batch* b) {
    const int count = (int)b->descs.size();
    std::vector<GInst> gi(count);
    std::vector<GShape> shp(count);
    // sizes: one allocation, carved in order; offsets first
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += al256(bytes); return o; };
    struct Off {
        size_t x, v, z, t, vp, yt, zacc, G, Gf, Rinv, part, flag;
        size_t q3, y3, gpart, gp, evals, uf, u64, lam, sweeps, w, U;
    };
    std::vector<Off> o(count);
    int64_t n_quant = 0, n_splitq = 0, n_xv = 0, n_xty = 0, n_dm = 0, n_gram = 0, n_reduce = 0, n_apply = 0;
    std::vector<int> c_quant(count), c_splitq(count), c_xv(count), c_xty(count), c_dm(count), c_gram(count),
        c_reduce(count), c_apply(count);
    std::vector<int> c_ygen32(count), c_ygen16(count), c_ychunks(count), c_gred(count), c_rayleigh(count),
        c_rotate(count), c_sign(count);
    int64_t n_pp = 0;
    b->any_f32 = false;
    b->any_vout = false;
    b->g_max_m = 0;
    for (int i = 0; i < count; ++i) {
        const ppca_instance_desc& ds = b->descs[i];
        GInst& g = gi[i];
        const int64_t n = ds.n, d = ds.d;
        const int m = ds.m;
        g.n = n;
        g.d = d;
        g.m = m;
        g.m_pad = (int)rup(m, 32);
        g.ldv = rup(d, 8);
        g.ldy = rup(n, 128);
        g.Dt = (int)cdiv(d, 128);
        g.nk = (int)cdiv(d, 64);
        g.ntiles = (int)(g.ldy / 128);
        g.kst = (int)(g.ldy / 64);
        // Z = X^T Y row groups of at most 8192 rows (128 K-stages): within the grouped
        // pass's fold interval (256), so each group's partial is one FP32 sum
        g.Sg = (int)cdiv(g.kst, 128);
        g.V0 = ds.V0;
        const bool f32 = ds.dtype == PPCA_F32;
        b->any_f32 |= f32;
        b->g_max_m = std::max(b->g_max_m, m);
        g.ld = f32 ? bf16_ld(d) : ds.ld;
        shp[i] = grouped_shape(d, m);
        g.gram_P = shp[i].gram_P;
        g.gram_T = shp[i].gram_T;
        g.gram_L = shp[i].gram_L;
        g.k = ds.k;
        g.xf32 = f32 ? 1 : 0;
        g.XP = ds.X;
        g.ldp = ds.ld;
        g.nparts = (int)cdiv(g.kst, kGramChunk);
        g.E = ds.E;
        g.lambda = ds.lambda;
        g.V_out = ds.V_out;
        b->any_vout |= ds.V_out != nullptr;
        // the BF16 copy of FP32 X serves the priming only: the pPCA step's Y pieces reuse it
        const size_t y3_bytes = (size_t)3 * g.m_pad * g.ldy * 2;
        const size_t xcopy = f32 ? (size_t)n * g.ld * 2 : 0;
        o[i].x = f32 ? take(std::max(xcopy, y3_bytes)) : 0;
        o[i].y3 = f32 ? o[i].x : take(y3_bytes);
        o[i].q3 = take((size_t)3 * g.m_pad * g.ldv * 2);
        o[i].gpart = take((size_t)g.nparts * g.m_pad * g.m_pad * 8);
        o[i].gp = take((size_t)m * m * 8);
        o[i].evals = take((size_t)m * 4);
        o[i].uf = take((size_t)m * m * 4);
        o[i].u64 = take((size_t)m * m * 8);
        o[i].lam = take((size_t)m * 8);
        o[i].sweeps = take(4);
        o[i].w = take((size_t)m * 8);
        o[i].U = take((size_t)m * m * 8);
        c_ygen32[i] = f32 ? g.ntiles : 0;
        c_ygen16[i] = f32 ? 0 : g.ntiles;
        c_ychunks[i] = g.nparts;
        c_gred[i] = (int)cdiv((int64_t)m * m, 256);
        c_rayleigh[i] = m;
        c_rotate[i] = (int)cdiv(d, 256) * ds.k;
        c_sign[i] = ds.k;
        for (int v : {c_ygen32[i], c_ygen16[i], c_ychunks[i], c_rotate[i]}) n_pp = std::max<int64_t>(n_pp, v);
        o[i].v = take((size_t)d * m * 4);
        o[i].z = take((size_t)d * m * 4);
        o[i].t = take((size_t)d * m * 4);
        o[i].vp = take((size_t)g.m_pad * g.ldv * 2);
        o[i].yt = take((size_t)g.m_pad * g.ldy * 2);
        o[i].zacc = take((size_t)g.Sg * g.m_pad * g.Dt * 128 * 4);
        o[i].G = take((size_t)m * m * 8);
        o[i].Gf = take((size_t)m * m * 4);
        o[i].Rinv = take((size_t)m * m * 4);
        o[i].part = take(gram_part_floats(d, m) * 4);
        o[i].flag = take(8);
        c_quant[i] = f32 ? (int)cdiv(n * (d / 8), 256) : 0;
        c_splitq[i] = (int)cdiv((int64_t)g.m_pad * g.ldv, 256);
        c_xv[i] = g.ntiles;
        c_xty[i] = g.Dt * g.Sg;
        c_dm[i] = (int)cdiv(d * m, 256);
        c_gram[i] = shp[i].gram_blocks;
        c_reduce[i] = shp[i].reduce_blocks;
        c_apply[i] = shp[i].apply_blocks;
        n_quant += c_quant[i];
        n_splitq += c_splitq[i];
        n_xv += c_xv[i];
        n_xty += c_xty[i];
        n_dm += c_dm[i];
        n_gram += c_gram[i];
        n_reduce += c_reduce[i];
        n_apply += c_apply[i];
    }
    const int64_t most = std::max({n_quant, n_splitq, n_xv, n_xty, n_dm, n_gram, n_reduce, n_apply});
    if (most >= (int64_t)1 << 31 || n_pp * count >= (int64_t)1 << 31) return false;
    const size_t tab_ints = (size_t)15 * (count + 1);
    const size_t o_tabs = take(tab_ints * 4);
    const size_t o_inst = take(sizeof(GInst) * count);
    const size_t o_maps = take(sizeof(GMaps) * count);
    const size_t o_x32 = take(sizeof(float*) * count);
    const size_t o_ld32 = take(sizeof(int64_t) * count);
    void* mem = nullptr;
    if (cudaMalloc(&mem, off) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int* st = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&st), 256) != cudaSuccess || cudaMemset(st, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(mem);
        if (st) cudaFree(st);
        return false;
    }
    char* base = static_cast<char*>(mem);
    std::vector<GMaps> maps(count);
    std::vector<const float*> x32(count);
    std::vector<int64_t> ld32(count);
    bool ok = true;
    for (int i = 0; i < count && ok; ++i) {
        const ppca_instance_desc& ds = b->descs[i];
        GInst& g = gi[i];
        g.X = ds.dtype == PPCA_F32 ? static_cast<const void*>(base + o[i].x) : ds.X;
        g.V = reinterpret_cast<float*>(base + o[i].v);
        g.Z = reinterpret_cast<float*>(base + o[i].z);
        g.T = reinterpret_cast<float*>(base + o[i].t);
        g.Vp = reinterpret_cast<__nv_bfloat16*>(base + o[i].vp);
        g.Yt = reinterpret_cast<__nv_bfloat16*>(base + o[i].yt);
        g.Zacc = reinterpret_cast<float*>(base + o[i].zacc);
        g.G = reinterpret_cast<double*>(base + o[i].G);
        g.Gf = reinterpret_cast<float*>(base + o[i].Gf);
        g.Rinv = reinterpret_cast<float*>(base + o[i].Rinv);
        g.gram_part = reinterpret_cast<float*>(base + o[i].part);
        g.flag = reinterpret_cast<int*>(base + o[i].flag);
        g.next = g.flag + 1;
        g.status = st;
        g.Q3 = reinterpret_cast<__nv_bfloat16*>(base + o[i].q3);
        g.Y3 = reinterpret_cast<__nv_bfloat16*>(base + o[i].y3);
        g.Gpart = reinterpret_cast<float2*>(base + o[i].gpart);
        g.Gp = reinterpret_cast<double*>(base + o[i].gp);
        g.evals = reinterpret_cast<float*>(base + o[i].evals);
        g.Uf = reinterpret_cast<float*>(base + o[i].uf);
        g.U64 = reinterpret_cast<double*>(base + o[i].u64);
        g.lam = reinterpret_cast<double*>(base + o[i].lam);
        g.sweeps = reinterpret_cast<int*>(base + o[i].sweeps);
        g.w = reinterpret_cast<double*>(base + o[i].w);
        g.U = reinterpret_cast<double*>(base + o[i].U);
        x32[i] = ds.dtype == PPCA_F32 ? static_cast<const float*>(ds.X) : nullptr;
        ld32[i] = ds.ld;
        ok = grouped_encode_maps(g, maps[i]) && grouped_encode_gram_maps(g, maps[i]);
    }
    std::vector<int> tabs;
    tabs.reserve(tab_ints);
    int* dtabs = reinterpret_cast<int*>(base + o_tabs);
    auto table = [&](const std::vector<int>& c) {
        GTable t;
        t.base = dtabs + tabs.size();
        t.count = count;
        int acc = 0;
        for (int v : c) {
            tabs.push_back(acc);
            acc += v;
        }
        tabs.push_back(acc);
        t.total = acc;
        return t;
    };
    b->t_quant = table(c_quant);
    b->t_splitq = table(c_splitq);
    b->t_xv = table(c_xv);
    b->t_xty = table(c_xty);
    b->t_dm = table(c_dm);
    b->t_gram = table(c_gram);
    b->t_reduce = table(c_reduce);
    b->t_apply = table(c_apply);
    b->t_ygen32 = table(c_ygen32);
    b->t_ygen16 = table(c_ygen16);
    b->t_ychunks = table(c_ychunks);
    b->t_gred = table(c_gred);
    b->t_rayleigh = table(c_rayleigh);
    b->t_rotate = table(c_rotate);
    b->t_sign = table(c_sign);
    if (ok)
        ok = cudaMemcpy(dtabs, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(base + o_inst, gi.data(), sizeof(GInst) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(base + o_maps, maps.data(), sizeof(GMaps) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(base + o_x32, x32.data(), sizeof(float*) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(base + o_ld32, ld32.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->g_done, cudaEventDisableTiming) == cudaSuccess;
    // the BF16 bases' padding (rows m..m_pad, columns d..ldv) stays zero for good
    for (int i = 0; i < count && ok; ++i)
        ok = cudaMemset(gi[i].Vp, 0, (size_t)gi[i].m_pad * gi[i].ldv * 2) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(mem);
        cudaFree(st);
        if (b->g_done) cudaEventDestroy(b->g_done);
        b->g_done = nullptr;
        return false;
    }
    b->g_mem = mem;
    b->g_status = st;
    b->g_inst = reinterpret_cast<GInst*>(base + o_inst);
    b->g_maps = reinterpret_cast<GMaps*>(base + o_maps);
    b->g_x32 = reinterpret_cast<const float* const*>(base + o_x32);
    b->g_ld32 = reinterpret_cast<const int64_t*>(base + o_ld32);
    b->g_host = std::move(gi);
    // the whole run is grouped: the slots' workspaces and BF16 priming copies go unused
    for (auto p : b->prime_buf) cudaFree(p);
    b->prime_buf.clear();
    for (auto* h : b->slots) {
        if (h->ws) cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_m = 0;
    }
    return true;
}

// CholeskyQR2 of every instance's src (V or Z) into dst (V or Z), through T (as
// run_orth; span_only: block power steps, each instance's second pass gated on
// its first pass's conditioning bound).
cudaError_t lockstep_orth(ppca_batch* b, int src, int dst, bool span_only = false) {
    const int count = (int)b->descs.size();
    cudaStream_t st = b->stream;
    cudaError_t e = grouped_gram(b->g_inst, b->t_gram, b->t_reduce, src, b->g_max_m, false, st);
    if (e == cudaSuccess) e = grouped_chol(b->g_inst, count, b->g_max_m, false, st, span_only);
    if (e == cudaSuccess) e = grouped_apply_rinv(b->g_inst, b->t_apply, src, kGT, b->g_max_m, st);
    if (e == cudaSuccess) e = grouped_gram(b->g_inst, b->t_gram, b->t_reduce, kGT, b->g_max_m, span_only, st);
    if (e == cudaSuccess) e = grouped_chol(b->g_inst, count, b->g_max_m, true, st, false, span_only);
    // the basis the next pass reads: its BF16 rounding written by the same kernel
    if (e == cudaSuccess) e = grouped_apply_rinv(b->g_inst, b->t_apply, kGT, dst, b->g_max_m, st, dst == kGV);
    return e;
}

// Enqueue (inside the capture) Algorithm 1 for every instance in lockstep on
// the batch stream: step 1 -- the BF16 rounding of FP32 X, V = orth(V0), then
// T times Z = X^T X V (fast BF16 pass), V = orth(Z) -- and steps 2-5.
ppca_status enqueue_lockstep(ppca_batch* b) {
    cudaStream_t st = b->stream;
    const int count = (int)b->descs.size();
    if (b->any_f32) CUDA_TRY(grouped_quantize_bf16(b->g_x32, b->g_ld32, b->g_inst, b->t_quant, st));
    CUDA_TRY(grouped_copy_v0(b->g_inst, b->t_dm, st));
    for (int i = 0; i < count; ++i)
        if (!b->descs[i].V0)
            CUDA_TRY(init_gaussian(b->g_host[i].V, b->descs[i].d, b->descs[i].m, b->descs[i].seed, st));
    CUDA_TRY(lockstep_orth(b, kGV, kGV));
    for (int t = 0; t < b->descs[0].T; ++t) {
        CUDA_TRY(grouped_xpass(b->g_inst, b->g_maps, b->t_xv, b->t_xty, b->t_dm, b->g_status, b->num_sms, st));
        CUDA_TRY(lockstep_orth(b, kGZ, kGV, /*span_only=*/true));
    }
    // steps 2-5 for every instance: Q = orth(V) (into Z), G = (X Q)^T (X Q) at
    // split precision on the data as given, the eigensolve, E = Q U[:, :k]
    if (b->any_vout) CUDA_TRY(grouped_copy_vout(b->g_inst, b->t_dm, st));
    CUDA_TRY(lockstep_orth(b, kGV, kGZ));
    CUDA_TRY(grouped_split_q(b->g_inst, b->t_splitq, st));
    CUDA_TRY(grouped_projected_gram(b->g_inst, b->g_maps, b->t_ygen32, b->t_ygen16, b->t_ychunks, b->t_gred,
                                    b->g_max_m, b->g_status, b->num_sms, st));
    CUDA_TRY(grouped_eigh(b->g_inst, count, b->t_rayleigh, b->g_max_m, st));
    CUDA_TRY(grouped_rotate(b->g_inst, b->t_rotate, b->t_sign, st));
    return PPCA_OK;
}

}  // namespace

extern "C" {

ppca_status ppca_batch_create(ppca_batch** out, const ppca_instance_desc* descs, int32_t count, int32_t slots,
                              void* stream) {
    if (!out) return fail(PPCA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!descs || count < 1) return fail(PPCA_ERR_INVALID, "need at least one instance");
    if (slots < 0) return fail(PPCA_ERR_INVALID, "slots < 0");
    const int nslots = std::min<int>(slots == 0 ? 8 : slots, count);
    for (int i = 0; i < count; ++i) {
        const ppca_instance_desc& ds = descs[i];
        ppca_status s = validate_x(ds.X, ds.n, ds.d, ds.ld, (ppca_dtype)ds.dtype, ds.row_scales);
        if (s != PPCA_OK) return fail(s, "instance %d: %s", i, g_last_error.c_str());
        const int64_t cap = std::min<int64_t>(std::min<int64_t>(ds.d, ds.n - 1), kMaxM);
        if (ds.m < 1 || ds.m > cap) return fail(PPCA_ERR_INVALID, "instance %d: m = %d out of range", i, ds.m);
        if (ds.k < 1 || ds.k > ds.m) return fail(PPCA_ERR_INVALID, "instance %d: k = %d out of range", i, ds.k);
        if (ds.T < 0) return fail(PPCA_ERR_INVALID, "instance %d: T < 0", i);
        if (!ds.E || !ds.lambda) return fail(PPCA_ERR_INVALID, "instance %d: NULL output", i);
    }
    ppca_batch* b = new (std::nothrow) ppca_batch();
    if (!b) return fail(PPCA_ERR_OOM, "host allocation failed");
    b->descs.assign(descs, descs + count);
    b->user_stream = static_cast<cudaStream_t>(stream);
    int device = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    b->num_sms = num_sms;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    for (int s = 0; s < nslots && e == cudaSuccess; ++s) {
        ppca_handle* h = new (std::nothrow) ppca_handle();
        if (!h) {
            free_batch(b);
            return fail(PPCA_ERR_OOM, "host allocation failed");
        }
        b->slots.push_back(h);
        h->device = device;
        h->num_sms = num_sms;
        h->sched.fused = 0;          // slots run concurrently: no cooperative launches
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
        b->slot_streams.push_back(st);
        h->stream = st;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        b->join.push_back(ev);
        e = cudaMalloc(reinterpret_cast<void**>(&h->status), 256);
        if (e == cudaSuccess) e = cudaMemset(h->status, 0, 256);
        // workspace for the largest instance of this slot
        int64_t nmax = 2, dmax = 1;
        int mmax = 1;
        for (int i = s; i < count; i += nslots) {
            nmax = std::max<int64_t>(nmax, descs[i].n);
            dmax = std::max<int64_t>(dmax, descs[i].d);
            mmax = std::max(mmax, (int)descs[i].m);
        }
        h->x = view_of(descs[s]);
        if (e == cudaSuccess) {
            ppca_status ps = ensure_workspace_dims(h, nmax, dmax, mmax);
            if (ps != PPCA_OK) {
                const std::string msg = g_last_error;
                free_batch(b);
                return fail(ps, "batch slot %d: %s", s, msg.c_str());
            }
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return fail(PPCA_ERR_CUDA, "batch setup failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return PPCA_OK;
}

ppca_status ppca_batch_run(ppca_batch* b) {
    if (!b) return fail(PPCA_ERR_INVALID, "batch is NULL");
    if (!b->exec) {
        const int nslots = (int)b->slots.size();
        b->grouped = lockstep_eligible(b) && prepare_lockstep(b);
        CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t launches0 = launches_so_far();
        ppca_status st = b->grouped ? enqueue_lockstep(b) : PPCA_OK;
        cudaError_t e = cudaEventRecord(b->fork, b->stream);
        for (int s = 0; s < nslots && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->slot_streams[s], b->fork, 0);
        for (size_t i = 0; i < b->descs.size() && e == cudaSuccess && st == PPCA_OK && !b->grouped; ++i) {
            const ppca_instance_desc& ds = b->descs[i];
            ppca_handle* h = b->slots[i % nslots];
            st = bind_instance(b, h, (int)(i % nslots), ds);
            if (st != PPCA_OK) break;
            ppca_prime_params prm;
            ppca_prime_params_default(&prm, PPCA_POWER);
            prm.V0 = ds.V0;
            prm.seed = ds.seed;
            prm.precision = PPCA_PREC_FAST;
            if (!b->inst_sched.empty()) h->sched = b->inst_sched[i];
            st = ppca_prime(h, PPCA_POWER, ds.m, ds.T, &prm);
            if (st == PPCA_OK) st = ppca_finalize(h, ds.k, ds.E, ds.lambda, PPCA_PREC_ACCURATE);
            if (st == PPCA_OK && ds.V_out) st = ppca_get_basis(h, ds.V_out);
            h->has_ref = false;
        }
        for (int s = 0; s < nslots && e == cudaSuccess; ++s) {
            e = cudaEventRecord(b->join[s], b->slot_streams[s]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[s], 0);
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
        if (st != PPCA_OK || e != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (st != PPCA_OK) return st;
            return fail(PPCA_ERR_CUDA, "batch capture failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : ee));
        }
        b->graph = g;
        b->kernels = launches_so_far() - launches0;
        CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    CUDA_TRY(cudaEventRecord(b->ev_in, b->user_stream));
    CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    CUDA_TRY(cudaEventRecord(b->ev_out, b->stream));
    CUDA_TRY(cudaStreamWaitEvent(b->user_stream, b->ev_out, 0));
    return PPCA_OK;
}

ppca_status ppca_batch_autotune(ppca_batch* b, int32_t reps, int32_t* groups) {
    if (!b) return fail(PPCA_ERR_INVALID, "batch is NULL");
    if (b->exec) return fail(PPCA_ERR_STATE, "the batch has already been captured");
    const int nslots = (int)b->slots.size();
    const int count = (int)b->descs.size();
    // group key: dtype, d, m, n rounded up to a power of two
    std::vector<std::pair<std::vector<int64_t>, int>> keys;     // key -> representative instance
    std::vector<int> group_of(count, -1);
    for (int i = 0; i < count; ++i) {
        const ppca_instance_desc& ds = b->descs[i];
        int64_t nb = 1;
        while (nb < ds.n) nb <<= 1;
        const std::vector<int64_t> key{ds.dtype, ds.d, ds.m, nb};
        int g = -1;
        for (size_t j = 0; j < keys.size(); ++j)
            if (keys[j].first == key) g = (int)j;
        if (g < 0) {
            g = (int)keys.size();
            keys.emplace_back(key, i);
        }
        group_of[i] = g;
    }
    std::vector<TcSchedule> best(keys.size());
    for (size_t g = 0; g < keys.size(); ++g) {
        const int i = keys[g].second;
        ppca_handle* h = b->slots[i % nslots];
        PPCA_TRY(bind_instance(b, h, i % nslots, b->descs[i]));       // tune on the priming data
        PPCA_TRY(autotune_handle(h, b->descs[i].m, 0, reps, false, &best[g]));
        h->has_ref = false;
    }
    b->inst_sched.resize(count);
    for (int i = 0; i < count; ++i) b->inst_sched[i] = best[group_of[i]];
    if (groups) *groups = (int32_t)keys.size();
    return PPCA_OK;
}

ppca_status ppca_batch_set_priming(ppca_batch* b, int32_t dtype) {
    if (!b) return fail(PPCA_ERR_INVALID, "batch is NULL");
    if (b->exec || !b->inst_sched.empty())
        return fail(PPCA_ERR_STATE, "set the priming data type before ppca_batch_autotune and the first run");
    if (dtype != PPCA_F32 && dtype != PPCA_BF16)
        return fail(PPCA_ERR_INVALID, "priming data type %d: PPCA_F32 or PPCA_BF16", (int)dtype);
    for (auto p : b->prime_buf) cudaFree(p);
    b->prime_buf.clear();
    b->prime_bf16 = dtype == PPCA_BF16;
    if (!b->prime_bf16) return PPCA_OK;
    const int nslots = (int)b->slots.size();
    for (int s = 0; s < nslots; ++s) {
        size_t bytes = 256;
        for (size_t i = s; i < b->descs.size(); i += nslots)
            if (b->descs[i].dtype == PPCA_F32)
                bytes = std::max(bytes, (size_t)b->descs[i].n * (size_t)bf16_ld(b->descs[i].d) * 2);
        void* p = nullptr;
        const cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (auto q : b->prime_buf) cudaFree(q);
            b->prime_buf.clear();
            b->prime_bf16 = false;
            return fail(PPCA_ERR_OOM, "cudaMalloc(%zu) for slot %d's BF16 priming copy failed", bytes, s);
        }
        b->prime_buf.push_back(p);
    }
    return PPCA_OK;
}

ppca_status ppca_batch_set_lockstep(ppca_batch* b, int32_t enable) {
    if (!b) return fail(PPCA_ERR_INVALID, "batch is NULL");
    if (b->exec) return fail(PPCA_ERR_STATE, "the batch has already been captured");
    b->lockstep = enable != 0;
    return PPCA_OK;
}

ppca_status ppca_batch_lockstep(const ppca_batch* b, int32_t* active) {
    if (!b || !active) return fail(PPCA_ERR_INVALID, "NULL argument");
    *active = b->grouped ? 1 : 0;
    return PPCA_OK;
}

ppca_status ppca_batch_kernel_count(const ppca_batch* b, int64_t* count) {
    if (!b || !count) return fail(PPCA_ERR_INVALID, "NULL argument");
    *count = b->kernels;
    return PPCA_OK;
}

ppca_status ppca_batch_sync(ppca_batch* b) {
    if (!b) return fail(PPCA_ERR_INVALID, "batch is NULL");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (b->g_status) PPCA_TRY(check_status_word(b->g_status));
    for (auto* h : b->slots) {
        ppca_status s = ppca_sync(h);
        if (s != PPCA_OK) return s;
    }
    return PPCA_OK;
}

ppca_status ppca_batch_destroy(ppca_batch* b) {
    free_batch(b);
    return PPCA_OK;
}

}  // extern "C"
