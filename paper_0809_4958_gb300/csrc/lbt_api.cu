// C ABI of the tracer-box library (declared in include/lbtracer.h).
//
// Host-side bookkeeping only: arena layout, box and chain tables, the ring of
// coarse boundary samples, step ordering and launches.  All arithmetic of the
// method runs in the kernels of lbt_kernels.cuh and lbt_synth.cu.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "lbt_fluct.cuh"
#include "lbt_internal.h"
#include "lbt_mlp.h"

using namespace lbt;

namespace {

thread_local std::string g_last_error;

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

size_t elem_bytes(int storage) { return storage == kF64 ? 8 : (storage == kF32 ? 4 : 2); }
size_t real_bytes(int storage) { return storage == kF64 ? 8 : 4; }

int validate_boxes(const lb_box_desc* boxes, int nboxes, int storage, std::string& why)
{
    if (!boxes || nboxes <= 0) {
        why = "no boxes";
        return LB_ERR_ARG;
    }
    if (storage < LB_STORE_F64 || storage > LB_STORE_BF16DEV) {
        why = "unknown storage";
        return LB_ERR_ARG;
    }
    for (int b = 0; b < nboxes; b++) {
        const lb_box_desc& d = boxes[b];
        char buf[160];
        if (d.E < 8 || d.E > 1024 || d.E % 8) {
            snprintf(buf, sizeof buf, "box %d: E=%d must be a multiple of 8 in [8, 1024]", b, d.E);
            why = buf;
            return LB_ERR_ARG;
        }
        if (!(d.tau > 0.5)) {
            snprintf(buf, sizeof buf, "box %d: tau=%g must exceed 1/2", b, d.tau);
            why = buf;
            return LB_ERR_ARG;
        }
        for (int a = 0; a < 3; a++) {
            const int m0 = d.face_mode[2 * a], m1 = d.face_mode[2 * a + 1];
            if (m0 != m1 || (m0 != LB_FACE_VELOCITY && m0 != LB_FACE_PERIODIC)) {
                snprintf(buf, sizeof buf, "box %d: faces of axis %d must both be VELOCITY or both PERIODIC", b, a);
                why = buf;
                return LB_ERR_ARG;
            }
        }
        if (d.time_interp != LB_TIME_LINEAR && d.time_interp != LB_TIME_HERMITE && d.time_interp != LB_TIME_MLP) {
            snprintf(buf, sizeof buf, "box %d: time_interp %d not available", b, d.time_interp);
            why = buf;
            return LB_ERR_ARG;
        }
        if (d.time_interp == LB_TIME_MLP) {
            if (d.K != 8 && d.K != 16) {
                snprintf(buf, sizeof buf, "box %d: the upsampler supports K = 8 or 16 (got %d)", b, d.K);
                why = buf;
                return LB_ERR_ARG;
            }
            for (int b2 = 0; b2 < b; b2++)
                if (boxes[b2].time_interp == LB_TIME_MLP && boxes[b2].K != d.K) {
                    why = "all upsampler boxes of a context share one K";
                    return LB_ERR_ARG;
                }
        }
        if (d.zoom < 0 || d.zoom > d.E - 1 || (d.zoom > 1 && d.time_interp == LB_TIME_MLP)) {
            snprintf(buf, sizeof buf, "box %d: zoom %d must be in [0, E-1]; the upsampler needs zoom 0 or 1", b,
                     d.zoom);
            why = buf;
            return LB_ERR_ARG;
        }
        if (d.frame_accel != 0 && d.frame_accel != 1) {
            snprintf(buf, sizeof buf, "box %d: frame_accel must be 0 or 1", b);
            why = buf;
            return LB_ERR_ARG;
        }
        if (d.K < 1 || d.nbeads < 0 || d.nbeads > kMaxBeads || !(d.rho_b > 0.0)) {
            snprintf(buf, sizeof buf, "box %d: need K >= 1, 0 <= nbeads <= %d, rho_b > 0", b, kMaxBeads);
            why = buf;
            return LB_ERR_ARG;
        }
    }
    return LB_OK;
}

Layout plan_layout(const lb_box_desc* boxes, int nboxes, int storage, int ring_slots)
{
    Layout L{};
    L.ring_slots = ring_slots;
    size_t off = 0;
    L.boxes = off;
    off = align_up(off + sizeof(BoxDev) * nboxes);
    L.tile_prefix = off;
    off = align_up(off + sizeof(int64_t) * (nboxes + 1));
    L.chains = off;
    off = align_up(off + sizeof(ChainDev) * nboxes);
    size_t pop = 0, ring = 0, zst = 0;
    int64_t beads = 0, chunks = 1;
    for (int b = 0; b < nboxes; b++) {
        const int64_t E = boxes[b].E, n3 = E * E * E;
        pop = align_up(pop + 19 * n3 * elem_bytes(storage));
        ring += align_up(6 * 3 * E * E * real_bytes(storage)) / real_bytes(storage);  // face sites
        if (boxes[b].zoom > 1) {
            const int64_t Ec = coarse_points(boxes[b].E, boxes[b].zoom);
            zst = align_up(zst + 6 * 3 * Ec * Ec * real_bytes(storage));
        }
        beads += boxes[b].nbeads;
        const int64_t c = (n3 + 4095) / 4096;
        if (c > chunks) chunks = c;
    }
    L.pop_bytes = pop;
    L.ring_slot_elems = ring;
    L.total_beads = beads;
    L.cons_chunks = chunks;
    L.pop_a = off;
    off = align_up(off + pop);
    L.pop_b = off;
    off = align_up(off + pop);
    L.ring = off;
    off = align_up(off + (size_t)ring_slots * ring * real_bytes(storage));
    L.zstage = off;
    L.zstage_bytes = zst;
    off = align_up(off + (zst > 0 ? zst : 16));
    L.pos = off;
    off = align_up(off + sizeof(double) * 3 * (beads + 1));
    L.vel = off;
    off = align_up(off + sizeof(double) * 3 * (beads + 1));
    L.forces = off;
    off = align_up(off + sizeof(ForceEntry) * 8 * (beads + 1));
    L.cons_partial = off;
    off = align_up(off + sizeof(double) * 4 * nboxes * chunks);
    L.cons_out = off;
    off = align_up(off + sizeof(double) * 8 * nboxes);
    L.status = off;
    off = align_up(off + sizeof(int32_t) * nboxes);
    L.step = off;
    off = align_up(off + sizeof(int64_t));
    L.tile_counter = off;
    off = align_up(off + sizeof(int64_t));
    L.faccel = off;  // frame-acceleration samples [box][ring slot][4]
    off = align_up(off + sizeof(double) * 4 * (size_t)nboxes * ring_slots);
    L.chain_accel = off;  // body acceleration of the step per chain [chain][4]
    off = align_up(off + sizeof(double) * 4 * (size_t)nboxes);
    L.fluct = off;  // fluctuating-collision parameters per box
    off = align_up(off + sizeof(FluctDev) * (size_t)nboxes);
    // upsampler: feature-set table, bf16 features and f32 outputs of all its boxes
    L.mlp_rows = 0;
    L.mlp_boxes = 0;
    L.mlp_K = 0;
    for (int b = 0; b < nboxes; b++)
        if (boxes[b].time_interp == LB_TIME_MLP) {
            L.mlp_rows += 6LL * boxes[b].E * boxes[b].E;
            L.mlp_boxes++;
            L.mlp_K = boxes[b].K;
        }
    L.mlp_sets = off;
    off = align_up(off + sizeof(MlpFeatureSet) * L.mlp_boxes);
    L.mlp_x = off;
    off = align_up(off + 2 * (size_t)kMlpIn * L.mlp_rows);
    L.mlp_y = off;
    off = align_up(off + 4 * (size_t)3 * L.mlp_K * L.mlp_rows);
    L.total = off;
    return L;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct lb_ctx {
    int storage = 0;
    int nboxes = 0;
    std::vector<lb_box_desc> desc;
    std::vector<BoxDev> boxes;
    std::vector<ChainDev> chains;      // one per box with nbeads > 0
    Layout L{};
    char* arena = nullptr;
    cudaStream_t stream = nullptr, side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool a_is_pop_a = true;            // which buffer holds the current state
    int64_t step = 0;                  // steps enqueued so far
    std::vector<int64_t> pushed;       // last boundary sample pushed per box (-1 none)
    std::vector<double> faccel_host;   // host copy of the frame-acceleration samples [box][slot][4]
    int kernel = LB_KERNEL_STAGED;
    int max_beads = 0;  // largest chain capacity of the context
    int sms = 0;        // multiprocessors of the context's device
    int bead_lanes = 0; // lanes per bead in the MD substeps (0 = default)
    int bead_bpt = 1;   // beads per MD thread
    double* hist = nullptr;  // chain trajectory ring (caller's device memory), lb_set_chain_history
    int hist_slots = 0;
    std::vector<size_t> zst_off;  // per zoomed box: byte offset of its coarse-sample staging (L.zstage)
    int threads = 256, ctas = 0, vw = 0;  // vw: sites per thread in stream-collide
    std::vector<int64_t> tile_prefix;  // for the current block size
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    bool graph_parity = true;
    bool profiling = false;
    int inject = LB_INJECT_NONE;            // test-only fault injection (lb_test_inject)
    int64_t wait_ns = kWaitLimitNs;         // limit of the stream-collide's bounded device waits
    const void* mlp_params = nullptr;  // bound upsampler parameters (device, caller-owned)
    double mlp_umax = 0.0;
    int64_t graph_step0 = 0;
    std::vector<cudaEvent_t> prof_ev;  // pairs around stream-collide launches
    size_t prof_used = 0;
    std::string err;

    template <class T>
    T* at(size_t off) const { return reinterpret_cast<T*>(arena + off); }
    void* curA() const { return arena + (a_is_pop_a ? L.pop_a : L.pop_b); }
    void* curB() const { return arena + (a_is_pop_a ? L.pop_b : L.pop_a); }
    bool has_velocity_faces(int b) const { return boxes[b].per_mask != 7; }
    int fail(int code, const std::string& msg)
    {
        err = msg;
        g_last_error = msg;
        return code;
    }
    int cuda_fail(cudaError_t e, const char* where)
    {
        return fail(LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    }
};

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
    } while (0)

namespace {

#define DISPATCH(storage, expr)                          \
    ((storage) == kF64   ? Launch<kF64>::expr            \
     : (storage) == kF32 ? Launch<kF32>::expr            \
     : (storage) == kF16 ? Launch<kF16>::expr            \
                         : Launch<kBF16>::expr)

int default_vw(int storage) { return storage == kF64 ? 2 : (storage == kF32 ? 4 : 8); }

int rebuild_tiles(lb_ctx* ctx)
{
    // sites per tile: fixed by the staged kernel's geometry, threads x sites per thread otherwise
    const int64_t T = ctx->kernel == LB_KERNEL_STAGED ? lbt_staged_tile_sites(ctx->vw)
                                                      : (int64_t)ctx->threads * ctx->vw;
    ctx->tile_prefix.assign(ctx->nboxes + 1, 0);
    for (int b = 0; b < ctx->nboxes; b++)
        ctx->tile_prefix[b + 1] = ctx->tile_prefix[b] + (ctx->boxes[b].n3 + T - 1) / T;
    CK(cudaMemcpyAsync(ctx->at<int64_t>(ctx->L.tile_prefix), ctx->tile_prefix.data(),
                       sizeof(int64_t) * (ctx->nboxes + 1), cudaMemcpyHostToDevice, ctx->stream));
    // the host vector must outlive the copy: synchronise (set-up path only)
    CK(cudaStreamSynchronize(ctx->stream));
    return LB_OK;
}

// Samples box b needs for the step that starts at step n.
void needed_samples(const lb_ctx* ctx, int b, int64_t n, int64_t& lo, int64_t& hi)
{
    const lb_box_desc& d = ctx->desc[b];
    const int64_t j = n / d.K;
    if (d.time_interp == LB_TIME_LINEAR) {
        lo = j;
        hi = j + 1;
    } else {
        lo = j > 0 ? j - 1 : 0;
        hi = j + 2;
    }
}

int check_samples(lb_ctx* ctx, int64_t n0, int64_t nsteps)
{
    for (int b = 0; b < ctx->nboxes; b++) {
        if (!ctx->has_velocity_faces(b)) continue;
        int64_t lo, hi;
        needed_samples(ctx, b, n0 + nsteps - 1, lo, hi);
        if (ctx->pushed[b] < hi) {
            char buf[200];
            snprintf(buf, sizeof buf, "box %d: step %lld needs boundary sample %lld, last pushed %lld", b,
                     (long long)(n0 + nsteps - 1), (long long)hi, (long long)ctx->pushed[b]);
            return ctx->fail(LB_ERR_STATE, buf);
        }
        int64_t lo0, hi0;
        needed_samples(ctx, b, n0, lo0, hi0);
        if (ctx->pushed[b] - ctx->L.ring_slots >= lo0) {
            char buf[200];
            snprintf(buf, sizeof buf, "box %d: sample %lld was overwritten before step %lld", b, (long long)lo0,
                     (long long)n0);
            return ctx->fail(LB_ERR_STATE, buf);
        }
    }
    return LB_OK;
}

// Box record with the body acceleration of the current step (reported fields)
BoxDev box_at_step(const lb_ctx* ctx, int box)
{
    BoxDev bd = ctx->boxes[box];
    double a[3];
    frame_accel_at(bd, ctx->faccel_host.data(), ctx->L.ring_slots, ctx->step, a);
    for (int c = 0; c < 3; c++) bd.accel[c] = a[c];
    return bd;
}

// Enqueue one step n -> n+1 for every box; swaps the buffers.  At the start
// of a coarse interval the upsampler boxes first get their residuals.
int enqueue_step(lb_ctx* ctx, int64_t n)
{
    const int nch = (int)ctx->chains.size();
    void* A = ctx->curA();
    void* B = ctx->curB();
    if (ctx->L.mlp_boxes > 0 && n % ctx->L.mlp_K == 0) {
        const size_t rb = real_bytes(ctx->storage);
        MlpFeatureSet* sets = ctx->at<MlpFeatureSet>(ctx->L.mlp_sets);
        CK(mlp_sets_from_ring(sets, ctx->L.mlp_boxes, ctx->at<BoxDev>(ctx->L.boxes), ctx->arena + ctx->L.ring,
                              (int64_t)(ctx->L.ring_slot_elems * rb), ctx->L.ring_slots, (int)rb,
                              ctx->at<int64_t>(ctx->L.step), ctx->stream));
        CK(mlp_features(sets, ctx->L.mlp_boxes, ctx->L.mlp_rows, ctx->mlp_umax, ctx->storage == kF64,
                        ctx->arena + ctx->L.mlp_x, ctx->stream));
        // residuals column-major (see SCParams::mlp_ystride); a timed-out MMA
        // flags the first upsampler box
        int first = 0;
        while (first < ctx->nboxes && ctx->boxes[first].mlp_row < 0) first++;
        CK(mlp_forward_tc(ctx->arena + ctx->L.mlp_x, ctx->L.mlp_rows, ctx->mlp_params, ctx->L.mlp_K,
                          ctx->at<float>(ctx->L.mlp_y), ctx->at<int32_t>(ctx->L.status) + first, ctx->stream,
                          ctx->L.mlp_rows));
    }
    if (nch > 0) {
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
        CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
        BeadParams bp;
        bp.A = A;
        bp.boxes = ctx->at<BoxDev>(ctx->L.boxes);
        bp.chains = ctx->at<ChainDev>(ctx->L.chains);
        bp.pos = ctx->at<double>(ctx->L.pos);
        bp.vel = ctx->at<double>(ctx->L.vel);
        bp.forces = ctx->at<ForceEntry>(ctx->L.forces);
        bp.faccel = ctx->at<double>(ctx->L.faccel);
        bp.chain_accel = ctx->at<double>(ctx->L.chain_accel);
        bp.ring_slots = ctx->L.ring_slots;
        bp.step = ctx->at<int64_t>(ctx->L.step);
        bp.status = ctx->at<int32_t>(ctx->L.status);
        bp.hist = ctx->hist;
        bp.hist_stride = 3 * (int64_t)ctx->L.total_beads;
        bp.hist_slots = ctx->hist_slots;
        bp.hist_pad = 0;
        CK(DISPATCH(ctx->storage, bead_couple(bp, nch, ctx->max_beads, ctx->bead_lanes, ctx->bead_bpt, ctx->side)));
        CK(cudaEventRecord(ctx->ev_join, ctx->side));
    }
    SCParams sp;
    sp.A = A;
    sp.B = B;
    sp.ring = ctx->arena + ctx->L.ring;
    sp.ring_slot_elems = (int64_t)ctx->L.ring_slot_elems;
    sp.ring_slots = ctx->L.ring_slots;
    sp.faccel = ctx->at<double>(ctx->L.faccel);
    sp.mlp_y = ctx->at<float>(ctx->L.mlp_y);
    sp.mlp_ystride = ctx->L.mlp_rows;
    sp.mlp_yunit = (float)(ctx->mlp_umax / kMlpOutDiv);
    sp.boxes = ctx->at<BoxDev>(ctx->L.boxes);
    sp.tile_prefix = ctx->at<int64_t>(ctx->L.tile_prefix);
    sp.general = 0;
    for (const BoxDev& bd : ctx->boxes) {
        if (bd.fluct) sp.general = 2;
        else if ((bd.per_mask != 0 || bd.has_accel) && sp.general == 0) sp.general = 1;
    }
    sp.fluct = ctx->at<FluctDev>(ctx->L.fluct);
    sp.nboxes = ctx->nboxes;
    sp.total_tiles = ctx->tile_prefix[ctx->nboxes];
    sp.step = ctx->at<int64_t>(ctx->L.step);
    sp.tile_counter = ctx->at<int64_t>(ctx->L.tile_counter);
    sp.status = ctx->at<int32_t>(ctx->L.status);
    sp.wait_ns = ctx->wait_ns;
    sp.withhold_tile = ctx->inject == LB_INJECT_WITHHOLD_LAST_TILE ? sp.total_tiles - 1 : -1;
    sp.hint_loads = nch > 0;
    sp.pad_hint = 0;
    const bool timed = ctx->profiling && ctx->prof_used + 2 <= ctx->prof_ev.size();
    // inside a stream capture the timing events must become event-record nodes of the graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (timed) CK(cudaStreamIsCapturing(ctx->stream, &cap));
    const unsigned evflags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (timed) CK(cudaEventRecordWithFlags(ctx->prof_ev[ctx->prof_used], ctx->stream, evflags));
    // The persistent stream-collide grid holds every SM (a block fills the
    // register file), so a bead block launched next to it would wait for the
    // whole sweep.  With few chains, leave one SM per chain to the bead kernel
    // so it runs alongside; with many chains the atomic tile counter balances
    // bead blocks and stream-collide blocks by itself.
    int ctas = ctx->ctas;
    if (ctas == 0 && ctx->kernel == LB_KERNEL_STAGED && nch > 0 && nch <= ctx->sms / 8) ctas = ctx->sms - nch;
    CK(DISPATCH(ctx->storage, stream_collide(sp, ctx->kernel, ctx->threads, ctas, ctx->vw, ctx->stream)));
    if (timed) {
        CK(cudaEventRecordWithFlags(ctx->prof_ev[ctx->prof_used + 1], ctx->stream, evflags));
        ctx->prof_used += 2;
    }
    if (nch > 0) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    ForcedParams fp;
    fp.A = A;
    fp.B = B;
    fp.boxes = ctx->at<BoxDev>(ctx->L.boxes);
    fp.chains = ctx->at<ChainDev>(ctx->L.chains);
    fp.forces = ctx->at<ForceEntry>(ctx->L.forces);
    fp.chain_accel = ctx->at<double>(ctx->L.chain_accel);
    fp.status = ctx->at<int32_t>(ctx->L.status);
    fp.step = ctx->at<int64_t>(ctx->L.step);
    fp.tile_counter = ctx->at<int64_t>(ctx->L.tile_counter);
    fp.nchains = nch;
    fp.splits = (8 * ctx->max_beads + kForcedThreads - 1) / kForcedThreads;
    if (fp.splits < 1) fp.splits = 1;
    CK(DISPATCH(ctx->storage, forced(fp, ctx->stream)));
    ctx->a_is_pop_a = !ctx->a_is_pop_a;
    return LB_OK;
}

int wait_stream(lb_ctx* ctx, int timeout_ms)
{
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return ctx->cuda_fail(e, "cudaStreamQuery");
        const auto ms =
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_ms >= 0 && ms > timeout_ms) return ctx->fail(LB_ERR_TIMEOUT, "stream wait timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return LB_OK;
}

int first_status(lb_ctx* ctx, int box)
{
    std::vector<int32_t> st(ctx->nboxes);
    CK(cudaMemcpyAsync(st.data(), ctx->at<int32_t>(ctx->L.status), sizeof(int32_t) * ctx->nboxes,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < ctx->nboxes; b++) {
        if ((box < 0 || box == b) && st[b] != 0) {
            char buf[96];
            snprintf(buf, sizeof buf, "box %d has status %d", b, st[b]);
            return ctx->fail(st[b], buf);
        }
    }
    return LB_OK;
}

constexpr int kDefaultTimeoutMs = 120000;

}  // namespace

void lbt_set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

extern "C" {

int32_t lb_plan(const lb_box_desc* boxes, int32_t nboxes, int32_t storage, int32_t ring_slots, size_t* arena_bytes)
{
    std::string why;
    int st = validate_boxes(boxes, nboxes, storage, why);
    if (st) {
        g_last_error = why;
        return st;
    }
    if (ring_slots == 0) ring_slots = kRingSlots;
    if (ring_slots < kRingSlots || ring_slots > kMaxRingSlots) {
        g_last_error = "ring_slots must be 0 (= 4) or in [4, 4096]";
        return LB_ERR_ARG;
    }
    if (!arena_bytes) {
        g_last_error = "null arena_bytes";
        return LB_ERR_ARG;
    }
    *arena_bytes = plan_layout(boxes, nboxes, storage, ring_slots).total;
    return LB_OK;
}

int32_t lb_create(const lb_box_desc* boxes, int32_t nboxes, int32_t storage, int32_t ring_slots, void* arena,
                  size_t arena_bytes, void* stream, lb_ctx** out)
{
    std::string why;
    int st = validate_boxes(boxes, nboxes, storage, why);
    if (st) {
        g_last_error = why;
        return st;
    }
    if (ring_slots == 0) ring_slots = kRingSlots;
    if (ring_slots < kRingSlots || ring_slots > kMaxRingSlots) {
        g_last_error = "ring_slots must be 0 (= 4) or in [4, 4096]";
        return LB_ERR_ARG;
    }
    if (!out || !arena) {
        g_last_error = "null arena or out";
        return LB_ERR_ARG;
    }
    Layout L = plan_layout(boxes, nboxes, storage, ring_slots);
    if (arena_bytes < L.total) {
        g_last_error = "arena smaller than lb_plan size";
        return LB_ERR_SIZE;
    }
    if (reinterpret_cast<uintptr_t>(arena) % kAlign) {
        g_last_error = "arena must be 256-byte aligned";
        return LB_ERR_ARG;
    }
    lb_ctx* ctx = new lb_ctx();
    ctx->storage = storage;
    ctx->nboxes = nboxes;
    ctx->desc.assign(boxes, boxes + nboxes);
    ctx->L = L;
    ctx->arena = reinterpret_cast<char*>(arena);
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    ctx->pushed.assign(nboxes, -1);
    ctx->faccel_host.assign((size_t)nboxes * ring_slots * 4, 0.0);
    ctx->vw = lbt_staged_default_spt(storage);  // the default kernel is the staged one
    ctx->threads = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_last_error = std::string("stream/event creation: ") + cudaGetErrorString(e);
        lb_destroy(ctx);
        return LB_ERR_CUDA;
    }
    // box and chain tables
    size_t pop = 0, ring = 0, zst = 0;
    ctx->zst_off.assign(nboxes, 0);
    int64_t beads = 0, mlp_rows = 0;
    std::vector<MlpFeatureSet> mlp_sets;
    for (int b = 0; b < nboxes; b++) {
        const lb_box_desc& d = boxes[b];
        BoxDev bd{};
        const int64_t E = d.E, n3 = E * E * E;
        bd.f_off = (int64_t)(pop / elem_bytes(storage));
        bd.n3 = n3;
        bd.ring_off = (int64_t)ring;
        bd.E = d.E;
        bd.zoom = d.zoom > 1 ? d.zoom : 1;
        bd.Ec = coarse_points(d.E, bd.zoom);
        bd.div_magic = ((1ull << 40) + (uint64_t)d.E - 1) / (uint64_t)d.E;
        bd.mlp_row = -1;
        if (d.time_interp == LB_TIME_MLP) {
            MlpFeatureSet fs{};
            fs.row_off = mlp_rows;
            fs.E = d.E;
            fs.box = b;
            bd.mlp_row = mlp_rows;
            mlp_sets.push_back(fs);
            mlp_rows += 6LL * d.E * d.E;
        }
        bd.per_mask = (d.face_mode[0] == LB_FACE_PERIODIC ? 1 : 0) | (d.face_mode[2] == LB_FACE_PERIODIC ? 2 : 0) |
                      (d.face_mode[4] == LB_FACE_PERIODIC ? 4 : 0);
        bd.time_interp = d.time_interp;
        bd.K = d.K;
        bd.chain = -1;
        bd.frame = d.frame_accel;
        bd.box = b;
        bd.tau = d.tau;
        bd.rho_b = d.rho_b;
        for (int a = 0; a < 3; a++) bd.accel[a] = d.body_accel[a];
        bd.has_accel =
            (d.frame_accel || d.body_accel[0] != 0.0 || d.body_accel[1] != 0.0 || d.body_accel[2] != 0.0) ? 1 : 0;
        if (d.nbeads > 0) {
            ChainDev ch{};
            ch.box = b;
            ch.nbeads = 0;
            ch.n_md = 1;
            ch.bead_off = beads;
            ch.force_off = 8 * beads;
            ch.mass = 1.0;
            bd.chain = (int)ctx->chains.size();
            ctx->chains.push_back(ch);
            if (d.nbeads > ctx->max_beads) ctx->max_beads = d.nbeads;
            beads += d.nbeads;
        }
        ctx->boxes.push_back(bd);
        pop = align_up(pop + 19 * n3 * elem_bytes(storage));
        ring += align_up(6 * 3 * n3 / E * real_bytes(storage)) / real_bytes(storage);  // 6 x 3 x E^2
        if (bd.zoom > 1) {
            ctx->zst_off[b] = zst;
            zst = align_up(zst + 6 * 3 * (size_t)bd.Ec * bd.Ec * real_bytes(storage));
        }
    }
    // zero the whole arena once (ring, status, step counter, force lists ...)
    e = cudaMemsetAsync(arena, 0, L.total, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->at<BoxDev>(L.boxes), ctx->boxes.data(), sizeof(BoxDev) * nboxes,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !ctx->chains.empty())
        e = cudaMemcpyAsync(ctx->at<ChainDev>(L.chains), ctx->chains.data(), sizeof(ChainDev) * ctx->chains.size(),
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !mlp_sets.empty())
        e = cudaMemcpyAsync(ctx->at<MlpFeatureSet>(L.mlp_sets), mlp_sets.data(), sizeof(MlpFeatureSet) * mlp_sets.size(),
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        g_last_error = std::string("arena set-up: ") + cudaGetErrorString(e);
        lb_destroy(ctx);
        return LB_ERR_CUDA;
    }
    if (rebuild_tiles(ctx) != LB_OK) {
        g_last_error = ctx->err;
        lb_destroy(ctx);
        return LB_ERR_CUDA;
    }
    *out = ctx;
    return LB_OK;
}

int32_t lb_destroy(lb_ctx* ctx)
{
    if (!ctx) return LB_OK;
    if (ctx->side) {
        wait_stream(ctx, kDefaultTimeoutMs);
        cudaStreamSynchronize(ctx->side);
    }
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (cudaEvent_t ev : ctx->prof_ev) cudaEventDestroy(ev);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    delete ctx;
    return LB_OK;
}

int32_t lb_init(lb_ctx* ctx, int32_t box, const void* u0)
{
    if (!ctx || !u0) return LB_ERR_ARG;
    if (box == LB_ALL_BOXES) {
        if (ctx->nboxes != 1) return ctx->fail(LB_ERR_ARG, "lb_init with all boxes needs one u0 per box; call per box");
        box = 0;
    }
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    if (ctx->nboxes > 1 && ctx->step > 0)
        return ctx->fail(LB_ERR_STATE, "boxes of a multi-box context are initialised before the first step");
    const BoxDev& bd = ctx->boxes[box];
    const size_t eb = elem_bytes(ctx->storage), rb = real_bytes(ctx->storage);
    void* A = reinterpret_cast<char*>(ctx->curA()) + bd.f_off * eb;
    const void* src = u0;
    if (!is_device_ptr(u0)) {
        void* stage = reinterpret_cast<char*>(ctx->curB()) + bd.f_off * eb;
        CK(cudaMemcpyAsync(stage, u0, 3 * (size_t)bd.Ec * bd.Ec * bd.Ec * rb, cudaMemcpyHostToDevice, ctx->stream));
        src = stage;
    }
    CK(DISPATCH(ctx->storage, init(A, ctx->boxes.data(), box, bd.n3, src, ctx->stream)));
    CK(cudaMemsetAsync(ctx->at<int32_t>(ctx->L.status) + box, 0, sizeof(int32_t), ctx->stream));
    if (ctx->nboxes == 1) {
        ctx->step = 0;
        CK(cudaMemsetAsync(ctx->at<int64_t>(ctx->L.step), 0, sizeof(int64_t), ctx->stream));
        ctx->pushed.assign(ctx->nboxes, -1);
    }
    return LB_OK;
}

int32_t lb_set_boundary(lb_ctx* ctx, int32_t box, int64_t j, const void* face_u)
{
    if (!ctx || !face_u) return LB_ERR_ARG;
    const size_t rb = real_bytes(ctx->storage);
    const int b0 = box == LB_ALL_BOXES ? 0 : box;
    const int b1 = box == LB_ALL_BOXES ? ctx->nboxes : box + 1;
    if (b0 < 0 || b1 > ctx->nboxes || b0 >= b1) return ctx->fail(LB_ERR_ARG, "box index out of range");
    for (int b = b0; b < b1; b++) {
        if (j != ctx->pushed[b] + 1) {
            char buf[160];
            snprintf(buf, sizeof buf, "box %d: boundary samples must be pushed in order (expected %lld, got %lld)", b,
                     (long long)(ctx->pushed[b] + 1), (long long)j);
            return ctx->fail(LB_ERR_STATE, buf);
        }
        int64_t lo, hi;
        needed_samples(ctx, b, ctx->step, lo, hi);
        if (j - ctx->L.ring_slots >= lo && j >= ctx->L.ring_slots) {
            char buf[160];
            snprintf(buf, sizeof buf, "box %d: sample %lld would overwrite sample %lld still needed at step %lld", b,
                     (long long)j, (long long)(j - ctx->L.ring_slots), (long long)ctx->step);
            return ctx->fail(LB_ERR_STATE, buf);
        }
    }
    char* slot = ctx->arena + ctx->L.ring + (size_t)(j % ctx->L.ring_slots) * ctx->L.ring_slot_elems * rb;
    const char* src = reinterpret_cast<const char*>(face_u);
    // boxes whose ring regions are packed back to back (and hold the samples
    // as given: no zoom) take one copy
    size_t packed = 0;
    bool contiguous = true;
    for (int b = b0; b < b1 && contiguous; b++) {
        contiguous = ctx->boxes[b].zoom == 1 &&
                     (size_t)ctx->boxes[b].ring_off * rb == (size_t)ctx->boxes[b0].ring_off * rb + packed;
        packed += 6 * 3 * (size_t)ctx->boxes[b].E * ctx->boxes[b].E * rb;
    }
    if (contiguous && b1 - b0 > 1) {
        CK(cudaMemcpyAsync(slot + ctx->boxes[b0].ring_off * rb, src, packed, cudaMemcpyDefault, ctx->stream));
        for (int b = b0; b < b1; b++) ctx->pushed[b] = j;
        return LB_OK;
    }
    for (int b = b0; b < b1; b++) {
        const BoxDev& bd = ctx->boxes[b];
        const int64_t Ec = bd.Ec;
        const size_t bytes = 6 * 3 * Ec * Ec * rb;
        if (bd.zoom == 1) {
            CK(cudaMemcpyAsync(slot + bd.ring_off * rb, src, bytes, cudaMemcpyDefault, ctx->stream));
        } else {
            // a zoomed box: the coarse sample into its staging, then bilinear in
            // space onto the face sites of the ring slot, once per sample, so
            // that a step interpolates only in time (Sec. 3: bilinear in space,
            // interpolated in time -- both linear, so the order is free)
            char* stage = ctx->arena + ctx->L.zstage + ctx->zst_off[b];
            CK(cudaMemcpyAsync(stage, src, bytes, cudaMemcpyDefault, ctx->stream));
            CK(DISPATCH(ctx->storage, upsample_faces(stage, slot + bd.ring_off * rb, bd.E, bd.Ec, bd.zoom, ctx->stream)));
        }
        src += bytes;
        ctx->pushed[b] = j;
    }
    return LB_OK;
}

int32_t lb_set_frame_accel(lb_ctx* ctx, int32_t box, int64_t sample_index, const double* a)
{
    if (!ctx || !a || sample_index < 0) return LB_ERR_ARG;
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    if (!ctx->boxes[box].frame) return ctx->fail(LB_ERR_ARG, "box was created without frame_accel");
    const int slot = (int)(sample_index % ctx->L.ring_slots);
    double* h = ctx->faccel_host.data() + ((size_t)box * ctx->L.ring_slots + slot) * 4;
    for (int c = 0; c < 3; c++) h[c] = a[c];
    h[3] = 0.0;
    // stream-ordered copy from pageable memory (staged when the call is made)
    CK(cudaMemcpyAsync(ctx->at<double>(ctx->L.faccel) + ((size_t)box * ctx->L.ring_slots + slot) * 4, h,
                       4 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    return LB_OK;
}

int32_t chain_couple(lb_ctx* ctx, int32_t box, const lb_chain_desc* d, const double* pos0, const double* vel0)
{
    if (!ctx || !d || !pos0) return LB_ERR_ARG;
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    const int ci = ctx->boxes[box].chain;
    if (ci < 0) return ctx->fail(LB_ERR_ARG, "box was planned without chain capacity (nbeads = 0)");
    if (ctx->boxes[box].fluct) return ctx->fail(LB_ERR_ARG, "chains couple to BGK boxes only");
    if (d->nbeads < 1 || d->nbeads > ctx->desc[box].nbeads || d->n_md < 1 || !(d->mass > 0) || d->kT < 0 ||
        !(d->R0 > 0) || d->zeta < 0 || d->pin_com < 0 || d->pin_com > 2 || d->eps < 0 ||
        (d->eps > 0 && !(d->sigma > 0)))
        return ctx->fail(LB_ERR_ARG, "invalid chain description");
    ChainDev& ch = ctx->chains[ci];
    ch.nbeads = d->nbeads;
    ch.n_md = d->n_md;
    ch.pin_com = d->pin_com;
    ch.k_fene = d->k_fene;
    ch.R0 = d->R0;
    ch.zeta = d->zeta;
    ch.mass = d->mass;
    ch.kT = d->kT;
    ch.eps = d->eps;
    ch.sigma = d->sigma;
    for (int a = 0; a < 3; a++) ch.f_ext[a] = d->f_ext[a];
    ch.seed = d->seed;
    {
        const double dt = 1.0 / d->n_md, skin = kBeadSkin, rl = std::sqrt(std::cbrt(2.0)) * d->sigma + skin;
        double* c = ch.md_d;
        c[kMdDt] = dt;
        c[kMdDtm] = dt / d->mass;
        c[kMdNamp] = d->kT > 0.0 ? std::sqrt(2.0 * d->kT * d->zeta / dt) : 0.0;
        c[kMdR02] = d->R0 * d->R0;
        c[kMdInvR02] = 1.0 / (d->R0 * d->R0);
        c[kMdKf] = d->k_fene;
        c[kMdZeta] = d->zeta;
        c[kMdSig2] = d->sigma * d->sigma;
        c[kMdRc2] = std::cbrt(2.0) * d->sigma * d->sigma;
        c[kMdE24] = 24.0 * d->eps;
        c[kMdRl2] = rl * rl;
        c[kMdHalfSkin2] = 0.25 * skin * skin;
        c[kMdInvN] = 1.0 / d->nbeads;
        c[kMdSkinComp2] = c[kMdHalfSkin2] / 3.0;
        for (int k = 0; k < kMdConsts; k++) ch.md_f[k] = (float)c[k];
        // FP32 derived constants rounded from their own FP32 operands, as the
        // device computed them before
        ch.md_f[kMdDt] = 1.0f / (float)d->n_md;
        ch.md_f[kMdDtm] = ch.md_f[kMdDt] / (float)d->mass;
        ch.md_f[kMdInvR02] = 1.0f / ch.md_f[kMdR02];
        ch.md_f[kMdRl2] = (float)rl * (float)rl;
    }
    const size_t bytes = sizeof(double) * 3 * d->nbeads;
    CK(cudaMemcpyAsync(ctx->at<double>(ctx->L.pos) + 3 * ch.bead_off, pos0, bytes, cudaMemcpyDefault, ctx->stream));
    if (vel0)
        CK(cudaMemcpyAsync(ctx->at<double>(ctx->L.vel) + 3 * ch.bead_off, vel0, bytes, cudaMemcpyDefault, ctx->stream));
    else
        CK(cudaMemsetAsync(ctx->at<double>(ctx->L.vel) + 3 * ch.bead_off, 0, bytes, ctx->stream));
    CK(cudaMemcpyAsync(ctx->at<ChainDev>(ctx->L.chains) + ci, &ch, sizeof(ChainDev), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the host copies above must not outlive this call
    return LB_OK;
}

int32_t lb_step(lb_ctx* ctx, int32_t nsteps)
{
    if (!ctx || nsteps < 0) return LB_ERR_ARG;
    if (nsteps == 0) return LB_OK;
    int st = check_samples(ctx, ctx->step, nsteps);
    if (st) return st;
    if (ctx->L.mlp_boxes > 0 && !ctx->mlp_params)
        return ctx->fail(LB_ERR_STATE, "upsampler boxes need parameters (lb_mlp_bind) before stepping");
    for (int k = 0; k < nsteps; k++) {
        st = enqueue_step(ctx, ctx->step);
        if (st) return st;
        ctx->step++;
    }
    return LB_OK;
}

int32_t lb_graph_capture(lb_ctx* ctx, int32_t nsteps)
{
    if (!ctx || nsteps <= 0 || nsteps % 2) return ctx ? ctx->fail(LB_ERR_ARG, "graph needs an even step count") : LB_ERR_ARG;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (ctx->L.mlp_boxes > 0) {
        if (!ctx->mlp_params) return ctx->fail(LB_ERR_STATE, "upsampler boxes need parameters (lb_mlp_bind)");
        if (nsteps % ctx->L.mlp_K || ctx->step % ctx->L.mlp_K)
            return ctx->fail(LB_ERR_ARG, "with upsampler boxes a graph covers whole coarse intervals from an interval start");
    }
    const bool parity = ctx->a_is_pop_a;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int st = LB_OK;
    for (int k = 0; k < nsteps && st == LB_OK; k++) st = enqueue_step(ctx, ctx->step + k);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->a_is_pop_a = parity;
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGraphInstantiate");
    // move the executable graph to the device now, so that the first launch
    // costs what every later one does
    e = cudaGraphUpload(ctx->graph, ctx->stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaGraphUpload");
    ctx->graph_steps = nsteps;
    ctx->graph_parity = parity;
    ctx->graph_step0 = ctx->step;
    return LB_OK;
}

int32_t lb_graph_launch(lb_ctx* ctx)
{
    if (!ctx || !ctx->graph) return ctx ? ctx->fail(LB_ERR_STATE, "no captured graph") : LB_ERR_ARG;
    if (ctx->a_is_pop_a != ctx->graph_parity) return ctx->fail(LB_ERR_STATE, "buffer parity differs from capture");
    if (ctx->L.mlp_boxes > 0 && (ctx->step - ctx->graph_step0) % ctx->L.mlp_K)
        return ctx->fail(LB_ERR_STATE, "graph with upsampler boxes launched away from an interval start");
    int st = check_samples(ctx, ctx->step, ctx->graph_steps);
    if (st) return st;
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    ctx->step += ctx->graph_steps;
    return LB_OK;
}

int32_t lb_read_fields(lb_ctx* ctx, int32_t box, int32_t what, void* dst)
{
    if (!ctx || !dst) return LB_ERR_ARG;
    const bool async = (what & LB_FIELD_ASYNC) != 0;
    what &= ~LB_FIELD_ASYNC;
    if (async && what == LB_FIELD_DEV && ctx->storage >= kF16 && !is_device_ptr(dst))
        return ctx->fail(LB_ERR_ARG, "asynchronous 16-bit population read-out needs a device destination");
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    const BoxDev& bd = ctx->boxes[box];
    const size_t eb = elem_bytes(ctx->storage), rb = real_bytes(ctx->storage);
    const bool dev = is_device_ptr(dst);
    const void* A = reinterpret_cast<const char*>(ctx->curA()) + bd.f_off * eb;
    if (what == LB_FIELD_CHAIN) {
        if (bd.chain < 0) return ctx->fail(LB_ERR_ARG, "box has no chain");
        const ChainDev& ch = ctx->chains[bd.chain];
        const size_t bytes = sizeof(double) * 3 * ch.nbeads;
        CK(cudaMemcpyAsync(dst, ctx->at<double>(ctx->L.pos) + 3 * ch.bead_off, bytes, cudaMemcpyDefault, ctx->stream));
        CK(cudaMemcpyAsync(reinterpret_cast<char*>(dst) + bytes, ctx->at<double>(ctx->L.vel) + 3 * ch.bead_off, bytes,
                           cudaMemcpyDefault, ctx->stream));
    } else if (what == LB_FIELD_RHO || what == LB_FIELD_U) {
        const size_t bytes = (what == LB_FIELD_RHO ? 1 : 3) * bd.n3 * rb;
        void* out = dev ? dst : reinterpret_cast<char*>(ctx->curB()) + bd.f_off * eb;  // staging in the free buffer
        const BoxDev bn = box_at_step(ctx, box);
        CK(DISPATCH(ctx->storage, fields(A, &bn, 0, bd.n3, what == LB_FIELD_RHO ? 0 : 1, out, ctx->stream)));
        if (!dev) CK(cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    } else if (what == LB_FIELD_DEV) {
        if (dev) {
            CK(DISPATCH(ctx->storage, read_dev(A, 19 * bd.n3, dst, ctx->stream)));
        } else if (ctx->storage == kF64 || ctx->storage == kF32) {
            CK(cudaMemcpyAsync(dst, A, 19 * bd.n3 * eb, cudaMemcpyDeviceToHost, ctx->stream));
        } else {
            // 16-bit storage: widen to float through the free buffer, 8 populations at a time
            char* stage = reinterpret_cast<char*>(ctx->curB()) + bd.f_off * eb;
            for (int i0 = 0; i0 < 19; i0 += 8) {
                const int ni = i0 + 8 <= 19 ? 8 : 19 - i0;
                const void* Ai = reinterpret_cast<const char*>(A) + (size_t)i0 * bd.n3 * eb;
                CK(DISPATCH(ctx->storage, read_dev(Ai, (int64_t)ni * bd.n3, stage, ctx->stream)));
                CK(cudaMemcpyAsync(reinterpret_cast<char*>(dst) + (size_t)i0 * bd.n3 * rb, stage, ni * bd.n3 * rb,
                                   cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
            }
        }
    } else {
        return ctx->fail(LB_ERR_ARG, "unknown field");
    }
    if (async) return LB_OK;
    int st = wait_stream(ctx, kDefaultTimeoutMs);
    if (st) return st;
    return first_status(ctx, box);
}

int32_t lb_conservation(lb_ctx* ctx, int32_t box, double* out)
{
    if (!ctx || !out) return LB_ERR_ARG;
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    CK(DISPATCH(ctx->storage,
                conservation(ctx->curA(), ctx->at<BoxDev>(ctx->L.boxes), ctx->at<ChainDev>(ctx->L.chains),
                             ctx->nboxes, ctx->L.cons_chunks, ctx->at<double>(ctx->L.vel),
                             ctx->at<double>(ctx->L.cons_partial), ctx->at<double>(ctx->L.cons_out),
                             ctx->at<int32_t>(ctx->L.status), ctx->stream)));
    double tmp[8];
    CK(cudaMemcpyAsync(tmp, ctx->at<double>(ctx->L.cons_out) + 8 * box, sizeof tmp, cudaMemcpyDeviceToHost, ctx->stream));
    int st = wait_stream(ctx, kDefaultTimeoutMs);
    if (st) return st;
    memcpy(out, tmp, 7 * sizeof(double));
    return first_status(ctx, box);
}

int32_t lb_vorticity(lb_ctx* ctx, int32_t box, int32_t lo, int32_t hi, double* out)
{
    if (!ctx || !out) return LB_ERR_ARG;
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    const BoxDev& bd = ctx->boxes[box];
    if (lo < 1 || hi > bd.E - 2 || lo > hi) return ctx->fail(LB_ERR_ARG, "the cube must lie inside sites 1 .. E-2");
    const size_t eb = elem_bytes(ctx->storage), rb = real_bytes(ctx->storage);
    const void* A = reinterpret_cast<const char*>(ctx->curA()) + bd.f_off * eb;
    // scratch in the box's region of the free buffer (19 E^3 elements): the
    // velocity field, then 512 block sums and the result
    char* stage = reinterpret_cast<char*>(ctx->curB()) + bd.f_off * eb;
    const size_t ubytes = (3 * (size_t)bd.n3 * rb + 255) / 256 * 256;
    double* sums = reinterpret_cast<double*>(stage + ubytes);
    const BoxDev bn = box_at_step(ctx, box);
    CK(DISPATCH(ctx->storage, fields(A, &bn, 0, bd.n3, 1, stage, ctx->stream)));
    CK(launch_vorticity(stage, ctx->storage == kF64, bd.E, lo, hi, sums, sums + 512, ctx->stream));
    double r = 0.0;
    CK(cudaMemcpyAsync(&r, sums + 512, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    int st = wait_stream(ctx, kDefaultTimeoutMs);
    if (st) return st;
    *out = r;
    return first_status(ctx, box);
}

int32_t lb_sync(lb_ctx* ctx, int32_t timeout_ms)
{
    if (!ctx) return LB_ERR_ARG;
    int st = wait_stream(ctx, timeout_ms);
    if (st) return st;
    return first_status(ctx, -1);
}

int32_t lb_status(lb_ctx* ctx, int32_t box, int32_t* status)
{
    if (!ctx || !status || box < 0 || box >= ctx->nboxes) return LB_ERR_ARG;
    int st = wait_stream(ctx, kDefaultTimeoutMs);
    if (st) return st;
    CK(cudaMemcpyAsync(status, ctx->at<int32_t>(ctx->L.status) + box, sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LB_OK;
}

int64_t lb_current_step(const lb_ctx* ctx) { return ctx ? ctx->step : -1; }

int32_t lb_set_launch(lb_ctx* ctx, int32_t kernel, int32_t threads, int32_t ctas, int32_t sites_per_thread)
{
    if (!ctx) return LB_ERR_ARG;
    const int dv = kernel == LB_KERNEL_STAGED ? lbt_staged_default_spt(ctx->storage) : default_vw(ctx->storage);
    const int vw = sites_per_thread == 0 ? dv : sites_per_thread;
    if (kernel == LB_KERNEL_STAGED) {
        if (threads != 0 || ctas < 0 || !lbt_staged_spt_ok(ctx->storage, vw))
            return ctx->fail(LB_ERR_ARG, "staged kernel: threads 0, ctas >= 0, sites_per_thread 0, 1 or "
                                         "(not FP64) 2");
    } else if (kernel == LB_KERNEL_REGISTER) {
        for (const BoxDev& bd : ctx->boxes)
            if (bd.fluct) return ctx->fail(LB_ERR_STATE, "the fluctuating collision runs in the staged kernel only");
        if (threads == 0) threads = 256;
        const int v4 = dv / 4 > 0 ? dv / 4 : 1;
        if (threads < 64 || threads > 256 || threads % 32 || ctas < 0 || (vw != dv && vw != dv / 2 && vw != v4))
            return ctx->fail(LB_ERR_ARG, "register kernel: threads multiple of 32 in [64, 256]; ctas >= 0; "
                                         "sites_per_thread the default, half or a quarter of it");
    } else {
        return ctx->fail(LB_ERR_ARG, "unknown stream-collide kernel");
    }
    ctx->kernel = kernel;
    ctx->threads = threads;
    ctx->ctas = ctas;
    ctx->vw = vw;
    if (kernel != LB_KERNEL_STAGED) {  // the injection exists in the staged kernel only
        ctx->inject = LB_INJECT_NONE;
        ctx->wait_ns = kWaitLimitNs;
    }
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return rebuild_tiles(ctx);
}

int32_t lb_set_chain_history(lb_ctx* ctx, void* dev, int32_t slots)
{
    if (!ctx) return LB_ERR_ARG;
    if (slots < 0 || (slots > 0 && !dev)) return ctx->fail(LB_ERR_ARG, "lb_set_chain_history: bad slots or buffer");
    if (slots > 0) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, dev) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            (reinterpret_cast<uintptr_t>(dev) & 7) != 0) {
            cudaGetLastError();
            return ctx->fail(LB_ERR_ARG, "lb_set_chain_history: the buffer must be 8-byte aligned device memory");
        }
        if (ctx->chains.empty()) return ctx->fail(LB_ERR_STATE, "lb_set_chain_history: the context has no chain");
    }
    ctx->hist = slots > 0 ? static_cast<double*>(dev) : nullptr;
    ctx->hist_slots = slots;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return LB_OK;
}

int32_t lb_set_bead_launch(lb_ctx* ctx, int32_t lanes, int32_t beads_per_thread)
{
    if (!ctx) return LB_ERR_ARG;
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8)
        return ctx->fail(LB_ERR_ARG, "lb_set_bead_launch: lanes must be 0, 1, 2, 4 or 8");
    if (beads_per_thread != 0 && beads_per_thread != 1 && beads_per_thread != 2)
        return ctx->fail(LB_ERR_ARG, "lb_set_bead_launch: beads_per_thread must be 0, 1 or 2");
    if (beads_per_thread == 2 && lanes != 1)
        return ctx->fail(LB_ERR_ARG, "lb_set_bead_launch: two beads per thread take one lane per bead");
    if (beads_per_thread == 0 && lanes != 2)
        return ctx->fail(LB_ERR_ARG, "lb_set_bead_launch: the chain-order layout (beads_per_thread 0) takes two lanes");
    if (beads_per_thread > 0 && lanes * ((ctx->max_beads + beads_per_thread - 1) / beads_per_thread) > 512)
        return ctx->fail(LB_ERR_ARG, "lb_set_bead_launch: lanes x beads per thread layout exceeds 512 threads");
    ctx->bead_lanes = lanes;
    ctx->bead_bpt = beads_per_thread;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return LB_OK;
}

// ---- checkpoint / restore ---------------------------------------------------
namespace {

constexpr uint64_t kCkptMagic = 0x3154504B4354424CULL;  // "LBTCKPT1" read as little-endian bytes
constexpr uint32_t kCkptVersion = 1;

// Fixed-size header at the start of a checkpoint.
struct CkptHeader {
    uint64_t magic;
    uint32_t version, storage;
    int32_t nboxes, ring_slots, nchains, pad;
    int64_t step;
    uint64_t desc_hash;   // FNV-1a of the box descriptions, field by field
    uint64_t total;       // bytes of the whole checkpoint
    uint64_t off_host, off_pop, off_ring, off_pos, off_vel, off_status, off_mlp_y;
    uint64_t bytes_pop, bytes_ring, bytes_beads, bytes_mlp_y;
};

struct CkptLayout {
    CkptHeader h;
    size_t host_bytes;  // pushed[nboxes] int64, faccel samples, chain records
};

void fnv(uint64_t& h, const void* p, size_t n)
{
    const unsigned char* b = reinterpret_cast<const unsigned char*>(p);
    for (size_t k = 0; k < n; k++) {
        h ^= b[k];
        h *= 1099511628211ULL;
    }
}

uint64_t desc_hash(const std::vector<lb_box_desc>& d)
{
    uint64_t h = 14695981039346656037ULL;
    for (const lb_box_desc& x : d) {
        fnv(h, &x.E, sizeof x.E);
        fnv(h, x.face_mode, sizeof x.face_mode);
        fnv(h, &x.time_interp, sizeof x.time_interp);
        fnv(h, &x.K, sizeof x.K);
        fnv(h, &x.nbeads, sizeof x.nbeads);
        fnv(h, &x.zoom, sizeof x.zoom);
        fnv(h, &x.frame_accel, sizeof x.frame_accel);
        fnv(h, &x.tau, sizeof x.tau);
        fnv(h, &x.rho_b, sizeof x.rho_b);
        fnv(h, x.body_accel, sizeof x.body_accel);
    }
    return h;
}

CkptLayout ckpt_layout(const lb_ctx* ctx)
{
    CkptLayout c{};
    CkptHeader& h = c.h;
    h.magic = kCkptMagic;
    h.version = kCkptVersion;
    h.storage = (uint32_t)ctx->storage;
    h.nboxes = ctx->nboxes;
    h.ring_slots = ctx->L.ring_slots;
    h.nchains = (int32_t)ctx->chains.size();
    h.step = ctx->step;
    h.desc_hash = desc_hash(ctx->desc);
    c.host_bytes = sizeof(int64_t) * ctx->nboxes + sizeof(double) * ctx->faccel_host.size() +
                   sizeof(ChainDev) * ctx->chains.size();
    h.bytes_pop = ctx->L.pop_bytes;
    h.bytes_ring = (size_t)ctx->L.ring_slots * ctx->L.ring_slot_elems * real_bytes(ctx->storage);
    h.bytes_beads = sizeof(double) * 3 * (size_t)ctx->L.total_beads;
    h.bytes_mlp_y = ctx->L.mlp_boxes > 0 ? sizeof(float) * 3 * (size_t)ctx->L.mlp_K * ctx->L.mlp_rows : 0;
    size_t off = align_up(sizeof(CkptHeader));
    h.off_host = off;
    off = align_up(off + c.host_bytes);
    h.off_pop = off;
    off = align_up(off + h.bytes_pop);
    h.off_ring = off;
    off = align_up(off + h.bytes_ring);
    h.off_pos = off;
    off = align_up(off + h.bytes_beads);
    h.off_vel = off;
    off = align_up(off + h.bytes_beads);
    h.off_status = off;
    off = align_up(off + sizeof(int32_t) * ctx->nboxes);
    h.off_mlp_y = off;
    off = align_up(off + h.bytes_mlp_y);
    h.total = off;
    return c;
}

}  // namespace

size_t lb_checkpoint_bytes(const lb_ctx* ctx) { return ctx ? ckpt_layout(ctx).h.total : 0; }

int32_t lb_save(lb_ctx* ctx, void* dst)
{
    if (!ctx || !dst) return LB_ERR_ARG;
    int st = wait_stream(ctx, kDefaultTimeoutMs);  // the state of every enqueued step
    if (st) return st;
    const CkptLayout c = ckpt_layout(ctx);
    const CkptHeader& h = c.h;
    std::vector<unsigned char> host(c.host_bytes);
    unsigned char* hp = host.data();
    memcpy(hp, ctx->pushed.data(), sizeof(int64_t) * ctx->nboxes);
    hp += sizeof(int64_t) * ctx->nboxes;
    memcpy(hp, ctx->faccel_host.data(), sizeof(double) * ctx->faccel_host.size());
    hp += sizeof(double) * ctx->faccel_host.size();
    if (!ctx->chains.empty()) memcpy(hp, ctx->chains.data(), sizeof(ChainDev) * ctx->chains.size());
    char* d = reinterpret_cast<char*>(dst);
    CK(cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyDefault, ctx->stream));
    if (c.host_bytes) CK(cudaMemcpyAsync(d + h.off_host, host.data(), c.host_bytes, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(d + h.off_pop, ctx->curA(), h.bytes_pop, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(d + h.off_ring, ctx->arena + ctx->L.ring, h.bytes_ring, cudaMemcpyDefault, ctx->stream));
    if (h.bytes_beads) {
        CK(cudaMemcpyAsync(d + h.off_pos, ctx->arena + ctx->L.pos, h.bytes_beads, cudaMemcpyDefault, ctx->stream));
        CK(cudaMemcpyAsync(d + h.off_vel, ctx->arena + ctx->L.vel, h.bytes_beads, cudaMemcpyDefault, ctx->stream));
    }
    CK(cudaMemcpyAsync(d + h.off_status, ctx->arena + ctx->L.status, sizeof(int32_t) * ctx->nboxes, cudaMemcpyDefault,
                       ctx->stream));
    if (h.bytes_mlp_y)
        CK(cudaMemcpyAsync(d + h.off_mlp_y, ctx->arena + ctx->L.mlp_y, h.bytes_mlp_y, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // host buffers above must outlive the copies
    return LB_OK;
}

int32_t lb_load(lb_ctx* ctx, const void* src)
{
    if (!ctx || !src) return LB_ERR_ARG;
    int st = wait_stream(ctx, kDefaultTimeoutMs);
    if (st) return st;
    const char* s = reinterpret_cast<const char*>(src);
    CkptHeader h{};
    CK(cudaMemcpyAsync(&h, s, sizeof h, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const CkptLayout c = ckpt_layout(ctx);
    if (h.magic != kCkptMagic || h.version != kCkptVersion)
        return ctx->fail(LB_ERR_ARG, "lb_load: not a checkpoint of this library (magic or version)");
    if ((int)h.storage != ctx->storage || h.nboxes != ctx->nboxes || h.ring_slots != ctx->L.ring_slots ||
        h.nchains != c.h.nchains || h.desc_hash != c.h.desc_hash || h.total != c.h.total)
        return ctx->fail(LB_ERR_ARG, "lb_load: the checkpoint was taken of a context with other boxes, storage or "
                                     "ring slots");
    if (h.step < 0) return ctx->fail(LB_ERR_ARG, "lb_load: negative step in the checkpoint");
    std::vector<unsigned char> host(c.host_bytes);
    if (c.host_bytes) CK(cudaMemcpyAsync(host.data(), s + h.off_host, c.host_bytes, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const unsigned char* hp = host.data();
    std::vector<int64_t> pushed(ctx->nboxes);
    memcpy(pushed.data(), hp, sizeof(int64_t) * ctx->nboxes);
    hp += sizeof(int64_t) * ctx->nboxes;
    std::vector<double> faccel(ctx->faccel_host.size());
    memcpy(faccel.data(), hp, sizeof(double) * faccel.size());
    hp += sizeof(double) * faccel.size();
    std::vector<ChainDev> chains(ctx->chains.size());
    if (!chains.empty()) memcpy(chains.data(), hp, sizeof(ChainDev) * chains.size());
    for (size_t k = 0; k < chains.size(); k++)  // the chain records must belong to the same boxes and capacities
        if (chains[k].box != ctx->chains[k].box || chains[k].bead_off != ctx->chains[k].bead_off ||
            chains[k].nbeads < 0 || chains[k].nbeads > ctx->desc[chains[k].box].nbeads)
            return ctx->fail(LB_ERR_ARG, "lb_load: chain records do not match the context");
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    CK(cudaMemcpyAsync(ctx->curA(), s + h.off_pop, h.bytes_pop, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(ctx->arena + ctx->L.ring, s + h.off_ring, h.bytes_ring, cudaMemcpyDefault, ctx->stream));
    if (h.bytes_beads) {
        CK(cudaMemcpyAsync(ctx->arena + ctx->L.pos, s + h.off_pos, h.bytes_beads, cudaMemcpyDefault, ctx->stream));
        CK(cudaMemcpyAsync(ctx->arena + ctx->L.vel, s + h.off_vel, h.bytes_beads, cudaMemcpyDefault, ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->arena + ctx->L.status, s + h.off_status, sizeof(int32_t) * ctx->nboxes, cudaMemcpyDefault,
                       ctx->stream));
    if (h.bytes_mlp_y)
        CK(cudaMemcpyAsync(ctx->arena + ctx->L.mlp_y, s + h.off_mlp_y, h.bytes_mlp_y, cudaMemcpyDefault, ctx->stream));
    if (!chains.empty())
        CK(cudaMemcpyAsync(ctx->at<ChainDev>(ctx->L.chains), chains.data(), sizeof(ChainDev) * chains.size(),
                           cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->at<double>(ctx->L.faccel), faccel.data(), sizeof(double) * faccel.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    const int64_t step = h.step, zero = 0;
    CK(cudaMemcpyAsync(ctx->at<int64_t>(ctx->L.step), &step, sizeof step, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->at<int64_t>(ctx->L.tile_counter), &zero, sizeof zero, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // host buffers above must outlive the copies
    ctx->step = step;
    ctx->pushed = pushed;
    ctx->faccel_host = faccel;
    ctx->chains = chains;
    return LB_OK;
}

int32_t lb_set_fluctuation(lb_ctx* ctx, int32_t box, double kT, uint64_t seed, const double* gamma)
{
    if (!ctx) return LB_ERR_ARG;
    if (box < 0 || box >= ctx->nboxes) return ctx->fail(LB_ERR_ARG, "box index out of range");
    BoxDev& bd = ctx->boxes[box];
    FluctDev fd{};
    if (gamma) {
        if (!(kT >= 0.0)) return ctx->fail(LB_ERR_ARG, "lb_set_fluctuation: kT must be >= 0");
        for (int k = 4; k < kQ; k++)
            if (!(gamma[k] > -1.0 && gamma[k] < 1.0))
                return ctx->fail(LB_ERR_ARG, "lb_set_fluctuation: gamma[4..18] must lie in (-1, 1)");
        if (bd.chain >= 0 || bd.has_accel)
            return ctx->fail(LB_ERR_ARG, "lb_set_fluctuation: boxes with a chain or a body force collide with BGK");
        if (ctx->kernel != LB_KERNEL_STAGED)
            return ctx->fail(LB_ERR_STATE, "lb_set_fluctuation: the fluctuating collision runs in the staged kernel");
        fd.seed = seed;
        fd.on = 1;
        for (int k = 4; k < kQ; k++) {
            // b_k = sum_i w_i e_k(c_i)^2; amplitude sqrt(mu b_k (1 - gamma_k^2)), mu = kT / c_s^2 = 3 kT
            const double b = bnorm36(k) / 36.0;
            fd.gamma[k - 4] = gamma[k];
            fd.amp[k - 4] = std::sqrt(3.0 * kT * b * (1.0 - gamma[k] * gamma[k]));
        }
    }
    bd.fluct = fd.on;
    CK(cudaMemcpyAsync(ctx->at<FluctDev>(ctx->L.fluct) + box, &fd, sizeof fd, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->at<BoxDev>(ctx->L.boxes) + box, &bd, sizeof bd, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // the host records above must outlive the copies
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return LB_OK;
}

int32_t lb_test_inject(lb_ctx* ctx, int32_t what, int32_t wait_limit_us)
{
    if (!ctx) return LB_ERR_ARG;
    if (what != LB_INJECT_NONE && what != LB_INJECT_WITHHOLD_LAST_TILE)
        return ctx->fail(LB_ERR_ARG, "lb_test_inject: unknown injection");
    if (wait_limit_us < 0 || wait_limit_us > 1000000)
        return ctx->fail(LB_ERR_ARG, "lb_test_inject: wait_limit_us must be in [0, 1000000]");
    if (what != LB_INJECT_NONE && ctx->kernel != LB_KERNEL_STAGED)
        return ctx->fail(LB_ERR_STATE, "lb_test_inject: the injection needs the staged stream-collide kernel");
    ctx->inject = what;
    ctx->wait_ns = wait_limit_us > 0 ? (int64_t)wait_limit_us * 1000 : kWaitLimitNs;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return LB_OK;
}

int32_t lb_profile(lb_ctx* ctx, int32_t enable, int32_t max_launches)
{
    if (!ctx || max_launches < 0) return LB_ERR_ARG;
    if (!enable) {
        ctx->profiling = false;
        return LB_OK;
    }
    for (cudaEvent_t ev : ctx->prof_ev) cudaEventDestroy(ev);
    ctx->prof_ev.assign(2 * (size_t)max_launches, nullptr);
    for (auto& ev : ctx->prof_ev) CK(cudaEventCreate(&ev));
    ctx->prof_used = 0;
    ctx->profiling = true;
    return LB_OK;
}

int32_t lb_profile_read(lb_ctx* ctx, double* total_ms, int64_t* launches)
{
    if (!ctx || !total_ms || !launches) return LB_ERR_ARG;
    int st = wait_stream(ctx, kDefaultTimeoutMs);
    if (st) return st;
    double sum = 0.0;
    for (size_t k = 0; k + 1 < ctx->prof_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->prof_ev[k], ctx->prof_ev[k + 1]));
        sum += ms;
    }
    *total_ms = sum;
    *launches = (int64_t)(ctx->prof_used / 2);
    return LB_OK;
}

const char* lb_last_error(const lb_ctx* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

size_t lb_synth_workspace_bytes(int32_t M, int32_t E)
{
    // phase table over 2E coordinates per axis: a zoomed coarse grid reaches at most E - 2 sites past the box
    return sizeof(double2) * 3 * (size_t)M * (size_t)(2 * E);
}

int32_t lb_synth_faces(const double* kvec, const double* amp, const double* omega, const double* phi, int32_t M,
                       int32_t E, int32_t zoom, int32_t K, int64_t j0, int64_t nsamp, int32_t out_dtype, void* out,
                       void* workspace, void* stream)
{
    if (!kvec || !amp || !omega || !phi || !out || !workspace || M < 1 || E < 2 || K < 1 || nsamp < 0 ||
        zoom < 1 || zoom > E - 1 || (out_dtype != LB_STORE_F64 && out_dtype != LB_STORE_F32)) {
        g_last_error = "lb_synth_faces: bad argument";
        return LB_ERR_ARG;
    }
    cudaError_t e = launch_synth_faces(kvec, amp, omega, phi, M, E, zoom, K, j0, nsamp, out_dtype == LB_STORE_F64,
                                       out, workspace, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        g_last_error = std::string("lb_synth_faces: ") + cudaGetErrorString(e);
        return e == cudaErrorInvalidValue ? LB_ERR_ARG : LB_ERR_CUDA;
    }
    return LB_OK;
}

int32_t lb_synth_volume(const double* kvec, const double* amp, const double* omega, const double* phi, int32_t M,
                        int32_t E, int32_t zoom, double t, int32_t out_dtype, void* out, void* workspace,
                        void* stream)
{
    if (!kvec || !amp || !omega || !phi || !out || !workspace || M < 1 || E < 2 || zoom < 1 || zoom > E - 1 ||
        (out_dtype != LB_STORE_F64 && out_dtype != LB_STORE_F32)) {
        g_last_error = "lb_synth_volume: bad argument";
        return LB_ERR_ARG;
    }
    cudaError_t e = launch_synth_volume(kvec, amp, omega, phi, M, E, zoom, t, out_dtype == LB_STORE_F64, out,
                                        workspace, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        g_last_error = std::string("lb_synth_volume: ") + cudaGetErrorString(e);
        return e == cudaErrorInvalidValue ? LB_ERR_ARG : LB_ERR_CUDA;
    }
    return LB_OK;
}

size_t lb_mlp_param_bytes(int32_t K) { return (K == 8 || K == 16) ? mlp_layout(K).bytes : 0; }

int32_t lb_mlp_bind(lb_ctx* ctx, const void* params, double u_max)
{
    if (!ctx || !params || !(u_max > 0)) return ctx ? ctx->fail(LB_ERR_ARG, "lb_mlp_bind: null parameters or u_max <= 0") : LB_ERR_ARG;
    if (ctx->L.mlp_boxes == 0) return ctx->fail(LB_ERR_ARG, "no box of this context uses the upsampler");
    ctx->mlp_params = params;
    ctx->mlp_umax = u_max;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return LB_OK;
}

size_t lb_mlp_train_bytes(int32_t K, int64_t batch_rows)
{
    if ((K != 8 && K != 16) || batch_rows < 1) return 0;
    return mlp_train_layout(K, batch_rows).bytes;
}

static int mlp_check(int32_t K, int64_t batch, const char* who)
{
    if ((K != 8 && K != 16) || batch < 1) {
        g_last_error = std::string(who) + ": K must be 8 or 16 and batch_rows >= 1";
        return LB_ERR_ARG;
    }
    return LB_OK;
}

static int cuda_status(cudaError_t e, const char* who)
{
    if (e == cudaSuccess) return LB_OK;
    g_last_error = std::string(who) + ": " + cudaGetErrorString(e);
    return LB_ERR_CUDA;
}

int32_t lb_mlp_train_init(void* ws, int32_t K, int64_t batch_rows, const float* master, void* stream)
{
    if (int st = mlp_check(K, batch_rows, "lb_mlp_train_init")) return st;
    if (!ws || !master) return LB_ERR_ARG;
    const MlpTrain W = mlp_train_layout(K, batch_rows);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* f = reinterpret_cast<float*>(ws);
    cudaError_t e = cudaMemcpyAsync(f + W.master, master, sizeof(float) * W.L.nmaster, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f + W.m, 0, sizeof(float) * W.L.nmaster, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f + W.v, 0, sizeof(float) * W.L.nmaster, s);
    if (e == cudaSuccess) e = mlp_export(f + W.master, K, reinterpret_cast<unsigned char*>(ws) + W.params_byte, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the master copy may come from pageable host memory
    return cuda_status(e, "lb_mlp_train_init");
}

int32_t lb_mlp_features(const void* s_prev, const void* s0, const void* s1, const void* s2, int32_t real_dtype,
                        int32_t E, double u_max, void* X, void* stream)
{
    if (!s_prev || !s0 || !s1 || !s2 || !X || E < 2 || !(u_max > 0) ||
        (real_dtype != LB_STORE_F64 && real_dtype != LB_STORE_F32)) {
        g_last_error = "lb_mlp_features: bad argument";
        return LB_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) {  // rows are written as 16-byte vectors
        g_last_error = "lb_mlp_features: X must be 16-byte aligned";
        return LB_ERR_ARG;
    }
    MlpFeatureSet fs{};
    fs.row_off = 0;
    fs.smp[0] = s_prev;
    fs.smp[1] = s0;
    fs.smp[2] = s1;
    fs.smp[3] = s2;
    fs.E = E;
    return cuda_status(mlp_features_one(fs, u_max, real_dtype == LB_STORE_F64, X, reinterpret_cast<cudaStream_t>(stream)),
                       "lb_mlp_features");
}

int32_t lb_mlp_targets(const void* s_prev, const void* s0, const void* s1, const void* s2, const void* fine,
                       int32_t real_dtype, int32_t E, int32_t K, int32_t first_interval, double u_max, float* T,
                       void* stream)
{
    if (!s_prev || !s0 || !s1 || !s2 || !fine || !T || E < 2 || K < 1 || !(u_max > 0) ||
        (real_dtype != LB_STORE_F64 && real_dtype != LB_STORE_F32)) {
        g_last_error = "lb_mlp_targets: bad argument";
        return LB_ERR_ARG;
    }
    const void* smp[4] = {s_prev, s0, s1, s2};
    return cuda_status(mlp_targets(smp, fine, E, K, first_interval, u_max, real_dtype == LB_STORE_F64, T,
                                   reinterpret_cast<cudaStream_t>(stream)),
                       "lb_mlp_targets");
}

int32_t lb_mlp_forward(const void* params, int32_t K, const void* X, int64_t rows, float* Y, void* stream)
{
    if (int st = mlp_check(K, 1, "lb_mlp_forward")) return st;
    if (!params || !X || !Y || rows < 0) return LB_ERR_ARG;
    return cuda_status(mlp_forward(X, rows, params, K, Y, reinterpret_cast<cudaStream_t>(stream)),
                       "lb_mlp_forward");
}

int32_t lb_mlp_grad(void* ws, int32_t K, int64_t batch_rows, const void* X, const float* T, int64_t rows,
                    float* grad_out, double* loss_out, void* stream)
{
    if (int st = mlp_check(K, batch_rows, "lb_mlp_grad")) return st;
    if (!ws || !X || !T || rows < 1 || rows > batch_rows) {
        g_last_error = "lb_mlp_grad: null pointer or rows outside [1, batch_rows]";
        return LB_ERR_ARG;
    }
    const MlpTrain W = mlp_train_layout(K, batch_rows);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = mlp_grad(reinterpret_cast<unsigned char*>(ws), W, X, T, rows, s);
    float* f = reinterpret_cast<float*>(ws);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, f + W.grad, sizeof(float) * W.L.nmaster, cudaMemcpyDefault, s);
    if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, f + W.loss, sizeof(double), cudaMemcpyDefault, s);
    return cuda_status(e, "lb_mlp_grad");
}

int32_t lb_mlp_train_step(void* ws, int32_t K, int64_t batch_rows, const void* X, const float* T, int64_t rows,
                          float lr, int64_t t, double* loss_out, void* stream)
{
    if (int st = mlp_check(K, batch_rows, "lb_mlp_train_step")) return st;
    if (!ws || !X || !T || rows < 1 || rows > batch_rows || t < 1 || !(lr > 0)) {
        g_last_error = "lb_mlp_train_step: bad argument";
        return LB_ERR_ARG;
    }
    const MlpTrain W = mlp_train_layout(K, batch_rows);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = mlp_grad(reinterpret_cast<unsigned char*>(ws), W, X, T, rows, s);
    if (e == cudaSuccess) e = mlp_adam(reinterpret_cast<unsigned char*>(ws), W, lr, t, s);
    if (e == cudaSuccess && loss_out)
        e = cudaMemcpyAsync(loss_out, reinterpret_cast<float*>(ws) + W.loss, sizeof(double), cudaMemcpyDefault, s);
    return cuda_status(e, "lb_mlp_train_step");
}

int32_t lb_mlp_export(const void* ws, int32_t K, int64_t batch_rows, void* params, void* stream)
{
    if (int st = mlp_check(K, batch_rows, "lb_mlp_export")) return st;
    if (!ws || !params) return LB_ERR_ARG;
    const MlpTrain W = mlp_train_layout(K, batch_rows);
    return cuda_status(cudaMemcpyAsync(params, reinterpret_cast<const char*>(ws) + W.params_byte, W.L.bytes,
                                       cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)),
                       "lb_mlp_export");
}

}  // extern "C"
