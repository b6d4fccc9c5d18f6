// Stream-collide with the boundary layer, staged through shared memory by
// TMA bulk copies (cp.async.bulk) in a warp-specialised pipeline.
//
// A tile is kSites consecutive sites of one box.  For population i the sites
// of a tile pull from one contiguous source range shifted by c_iy E + c_iz E^2
// (and by c_ix inside the row), so one bulk copy per population, widened by a
// 16-byte halo on each side for the x shift, brings everything the tile needs
// into shared memory; the x shift becomes an offset into that row.
//
// One producer warp claims tiles from a global counter and issues their 19
// copies into a ring of stages; a "full" barrier per stage counts the bytes
// landing, an "empty" barrier counts the consumer warps done with the stage.
// Fifteen consumer warps take the stages in order.  A consumer warp loads its
// sites' populations from the stage into registers and releases the stage at
// once, then collides and stores straight to global memory, so the copies of
// a later tile into that stage overlap the arithmetic and the stores of this
// one.  No block-wide barrier is taken inside the loop.
//
// Only sites whose pull source crosses a periodic face (a wrap) read global
// memory directly.  Copies are clamped to the box's arrays; sites whose
// source lies outside are boundary sites, which are overwritten with the
// boundary equilibrium anyway.
#pragma once
#include "lbt_device.cuh"

namespace lbt {

constexpr int kStagedHaloBytes = 16;  // x-shift halo on each side of a row
constexpr int kStagedConsumerWarps = 15;  // + the producer: four warps per scheduler
constexpr int kStagedConsumers = kStagedConsumerWarps * 32;
constexpr int kStagedThreads = kStagedConsumers + 32;  // + the producer warp
constexpr int kStagedHeaderBytes = 4096;               // barriers and tile headers
constexpr int kStagedMaxStages = 6;

// Tile geometry for SPT sites per consumer thread.  As many stages as fit in
// the 227 KB of shared memory a block may use (at most six).
template <int ST, int SPT>
struct Staged {
    using E = typename Stor<ST>::E;
    static constexpr int kSites = kStagedConsumers * SPT;
    static constexpr int kRowBytes = kSites * (int)sizeof(E);               // one population row of a tile
    static constexpr int kRowStride = kRowBytes + 2 * kStagedHaloBytes;
    static constexpr int kStageBytes = kQ * kRowStride;
    static constexpr int kFit = (227 * 1024 - kStagedHeaderBytes) / kStageBytes;
    static constexpr int kStages = kFit > kStagedMaxStages ? kStagedMaxStages : kFit;
    static constexpr int kSmemBytes = kStagedHeaderBytes + kStages * kStageBytes;
    static constexpr int kHalo = kStagedHaloBytes / (int)sizeof(E);         // halo elements
    static_assert(kStages >= 2, "tile too large for a two-stage pipeline");
    static_assert(kRowStride % 16 == 0, "bulk copies need 16-byte aligned rows");
};

// Sites per consumer thread the staged kernel supports per storage format
// (the first is the default): FP64 1; FP32 2 or 1; 16-bit 2 or 1.
inline bool staged_spt_ok(int storage, int spt) { return spt == 1 || (spt == 2 && storage != kF64); }
inline int staged_default_spt(int storage) { return storage == kF64 ? 1 : 2; }
inline int staged_tile_sites(int spt) { return kStagedConsumers * spt; }

// ---- PTX helpers (mbarrier + bulk copy) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Test the phase; a thread that finds it incomplete may be suspended in
// hardware for up to 20 us (or until the phase completes) instead of spinning
// and taking issue slots from the warps that compute.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase), "r"(20000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase of the barrier, giving up after limit_ns nanoseconds (one
// second by default; shorter only when a test makes a wait run out on purpose).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int64_t limit_ns)
{
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase))
        if (global_ns() - t0 > (uint64_t)limit_ns) return false;
    return true;
}

__device__ __forceinline__ int locate_box(const SCParams& p, int64_t tile)
{
    int lo = 0, hi = p.nboxes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.tile_prefix[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Shared-memory header: full and empty barriers, then the tile header the
// producer writes for each stage before it arms the barrier: the box record,
// first site, frozen flag, and what the collision and the boundary layer of
// the box need at this step -- BGK constants in the arithmetic type, the ring
// slots and weights of the time interpolation, the upsampler substep -- so
// that they are worked out (64-bit divisions, FP64 conversions, global loads)
// once per tile by the producer, not once per consumer warp.
template <int ST>
struct StagedTile {
    using A = typename Stor<ST>::A;
    using R = typename Stor<ST>::R;
    BoxDev bd;
    int64_t s0;
    int32_t box;
    int32_t mlp_s;
    int32_t frozen;  // the box carries an error status: its state does not change
    int32_t slot[4];
    R c[4];
    A om, om1, srcfac, drho_b;  // 1/tau, 1 - 1/tau, 1 - 1/(2 tau), rho_b - 1
};
// Consumers keep reading a tile's header after they have released its data
// stage (early release), so headers live in a ring of twice the stages: tile
// k uses header k mod 2S, which the producer rewrites for tile k + 2S only
// after every consumer warp has released tile k + S -- that is, after each of
// them has finished tile k (a warp takes the tiles in order).
template <int ST>
struct StagedHeader {
    uint64_t full[kStagedMaxStages];
    uint64_t empty[kStagedMaxStages];
    StagedTile<ST> t[2 * kStagedMaxStages];
};
static_assert(sizeof(StagedHeader<kF64>) <= kStagedHeaderBytes, "header does not fit");
static_assert(sizeof(StagedHeader<kF32>) <= kStagedHeaderBytes, "header does not fit");

// Producer (one thread): bulk copies of the 19 source rows of a tile.
template <int ST, int SPT>
__device__ __forceinline__ void issue_tile(const SCParams& p, const BoxDev& bd, int64_t s0, unsigned char* stage,
                                           uint64_t* bar)
{
    using E = typename Stor<ST>::E;
    constexpr int T = Staged<ST, SPT>::kSites, H = Staged<ST, SPT>::kHalo;
    const int64_t n3 = bd.n3, Ei = bd.E;
    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    int64_t lo[kQ], hi[kQ];
    uint32_t total = 0;
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const int64_t start = s0 - (cvec(i, 1) * Ei + cvec(i, 2) * Ei * Ei) - H;
        lo[i] = start > 0 ? start : 0;
        hi[i] = start + T + 2 * H < n3 ? start + T + 2 * H : n3;
        if (hi[i] > lo[i]) total += (uint32_t)((hi[i] - lo[i]) * sizeof(E));
    }
    mbar_arrive_expect_tx(bar, total);
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        if (hi[i] <= lo[i]) continue;
        const int64_t start = s0 - (cvec(i, 1) * Ei + cvec(i, 2) * Ei * Ei) - H;
        bulk_load(stage + i * Staged<ST, SPT>::kRowStride + (lo[i] - start) * sizeof(E), Ab + (int64_t)i * n3 + lo[i],
                  (uint32_t)((hi[i] - lo[i]) * sizeof(E)), bar);
    }
}

// Quotient and remainder of a site index by E with a precomputed multiplier:
// q = (s * m) >> 40 with m = ceil(2^40 / E), exact for s < 2^31 and E <= 1024.
__device__ __forceinline__ int div_e(int64_t s, uint64_t m) { return (int)(((uint64_t)s * m) >> 40); }

// Consumer thread c (0 .. 479) of one tile: sites s0 + c + k 480, so the lanes
// of a warp read consecutive shared-memory words and store consecutive global
// words.  Populations go to registers, the warp releases the stage, then the
// collision (BGK with the equilibrium of opposite pairs shared: the even part
// in c.u is common, the odd part changes sign) and the stores.
template <int ST, int SPT, bool PER, bool ACCEL>
__device__ __forceinline__ void staged_tile(const SCParams& p, const StagedTile<ST>& th, const unsigned char* stage,
                                            uint64_t* empty)
{
    using S = Stor<ST>;
    using E = typename S::E;
    using A = typename S::A;
    using R = typename S::R;
    constexpr int H = Staged<ST, SPT>::kHalo;
    constexpr int C = kStagedConsumers;
    const int tid = threadIdx.x;
    // site indices of a box fit 32 bits (E <= 1024)
    const int s0 = (int)th.s0;
    const BoxDev& bd = th.bd;

    const int Ei = bd.E;
    const int n3 = (int)bd.n3;
    // body acceleration of the step in the arithmetic type, converted once
    A acA[3] = {A(0), A(0), A(0)};
    if (ACCEL)
        for (int c = 0; c < 3; c++) acA[c] = (A)bd.accel[c];
    const uint64_t mE = bd.div_magic;
    const int per = bd.per_mask;
    const bool px = per & 1, py = per & 2, pz = per & 4;
    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;

    // coordinates of site k (recomputed where needed rather than held in
    // registers across the population loads)
    auto coords = [&](int k, int& x, int& y, int& z) {
        const int s = s0 + tid + k * C;
        const int sc = s < n3 ? s : 0;
        const int row = div_e(sc, mE);
        x = sc - row * Ei;
        z = div_e(row, mE);
        y = row - z * Ei;
    };
    int xs_[SPT], ys_[SPT], zs_[SPT];
    bool act[SPT], bnd[SPT];
    bool any_bnd = false;
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        act[k] = s0 + tid + k * C < n3;
        int x, y, z;
        coords(k, x, y, z);
        xs_[k] = x;
        ys_[k] = y;
        zs_[k] = z;
        bnd[k] = act[k] && ((!px && (x == 0 || x == Ei - 1)) || (!py && (y == 0 || y == Ei - 1)) ||
                            (!pz && (z == 0 || z == Ei - 1)));
        any_bnd |= bnd[k];
    }

    // f_i pulled into site k: shared memory, or global memory across a periodic
    // wrap; zero where it is not used (boundary and inactive sites)
    A f[kQ][SPT];
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        const E* row = reinterpret_cast<const E*>(stage + i * Staged<ST, SPT>::kRowStride);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            A v = S::in(row[H + tid + k * C - cx]);
            if (PER) {
                const int xs = xs_[k] - cx, ys = ys_[k] - cy, zs = zs_[k] - cz;
                const bool wrap = (px && (xs < 0 || xs >= Ei)) || (py && (ys < 0 || ys >= Ei)) ||
                                  (pz && (zs < 0 || zs >= Ei));
                if (wrap && act[k])
                    v = S::in(Ab[(int64_t)i * n3 + ((int64_t)wrapi(zs, Ei) * Ei + wrapi(ys, Ei)) * Ei + wrapi(xs, Ei)]);
            }
            f[i][k] = (act[k] && !bnd[k]) ? v : A(0);
        }
    }
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(empty);  // this warp is done with the stage

    A drho[SPT], ux[SPT], uy[SPT], uz[SPT];
    bool nonfinite = false;  // a density that is not finite or not positive
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        A r = A(0), jx = A(0), jy = A(0), jz = A(0);
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            r += f[i][k];
            if (cvec(i, 0)) jx += cvec(i, 0) * f[i][k];
            if (cvec(i, 1)) jy += cvec(i, 1) * f[i][k];
            if (cvec(i, 2)) jz += cvec(i, 2) * f[i][k];
        }
        const A rho = A(1) + r;
        nonfinite |= !(rho > A(0) && rho < A(1e30));  // NaN fails both comparisons
        const A inv = A(1) / rho;
        if (ACCEL) {
            jx += A(0.5) * rho * acA[0];
            jy += A(0.5) * rho * acA[1];
            jz += A(0.5) * rho * acA[2];
        }
        drho[k] = r;
        ux[k] = jx * inv;
        uy[k] = jy * inv;
        uz[k] = jz * inv;
    }
    // flag the box (it freezes from the next step on); boundary and inactive
    // sites pulled zeros, so only collided sites can raise the flag
    if (__any_sync(0xffffffffu, nonfinite) && (tid & 31) == 0) atomicCAS(&p.status[th.box], 0, LB_ERR_NONFINITE);
    // boundary sites: equilibrium of the boundary velocity from the ring
    if (any_bnd) {
        TimeWeights<R> tw;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            tw.slot[a] = th.slot[a];
            tw.c[a] = th.c[a];
        }
        const R* ring = reinterpret_cast<const R*>(p.ring);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            if (bnd[k]) {
                int pp, qq, x, y, z;
                if (PER) {
                    x = xs_[k];
                    y = ys_[k];
                    z = zs_[k];
                } else {
                    coords(k, x, y, z);
                }
                const int fc = owning_face(x, y, z, Ei, per, pp, qq);
                float res[3];
                load_mlp_residual(p, bd, th.mlp_s, fc, pp, qq, res);
                R ub[3];
                boundary_velocity<R>(ring, p.ring_slot_elems, bd, fc, pp, qq, tw, ub);
                add_mlp_residual<R>(p, bd, res, ub);
                drho[k] = th.drho_b;
                ux[k] = (A)ub[0];
                uy[k] = (A)ub[1];
                uz[k] = (A)ub[2];
            }
        }
    }
    const A om = th.om, om1 = th.om1, srcfac = th.srcfac;
    A usq[SPT], rho_[SPT], ua[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        usq[k] = A(1.5) * (ux[k] * ux[k] + uy[k] * uy[k] + uz[k] * uz[k]);
        rho_[k] = A(1) + drho[k];
        if (ACCEL) ua[k] = ux[k] * acA[0] + uy[k] * acA[1] + uz[k] * acA[2];
    }
    // post-collision value of population i at site k from its equilibrium deviation
    // populations are written in order 0, 1, ..., 18 through one running
    // pointer (row of population i at this thread's first site)
    E* out = Bb + s0 + tid;
    auto emit = [&](int i, int k, A deq, A cu) {
        A val = deq;
        if (!bnd[k]) {
            val = om1 * f[i][k] + om * deq;
            if (ACCEL) {
                const A w = wgt<A>(i);
                A ca = A(0);  // c_i . a in the arithmetic type (FP64 is slow on this part)
                if (cvec(i, 0)) ca += cvec(i, 0) * acA[0];
                if (cvec(i, 1)) ca += cvec(i, 1) * acA[1];
                if (cvec(i, 2)) ca += cvec(i, 2) * acA[2];
                val += srcfac * w * rho_[k] * (A(3) * (ca - ua[k]) + A(9) * cu * ca);
            }
        }
        // population 0 and odd i at `out`, the even partner of a pair one row further
        const int row = (i > 0 && (i & 1) == 0) ? n3 : 0;
        if (act[k]) out[row + k * C] = S::out(val);
    };
#pragma unroll
    for (int k = 0; k < SPT; k++) emit(0, k, wgt<A>(0) * (drho[k] - rho_[k] * usq[k]), A(0));
    // opposite pairs (1,2), (3,4), ..., (17,18)
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
        out += i == 1 ? n3 : 2 * n3;  // row of population i; population i + 1 is one row further
        const A w = wgt<A>(i);
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            A cu = A(0);
            if (cx) cu += cx * ux[k];
            if (cy) cu += cy * uy[k];
            if (cz) cu += cz * uz[k];
            const A even = w * (drho[k] + rho_[k] * (A(4.5) * cu * cu - usq[k]));
            const A odd = (A(3) * w) * rho_[k] * cu;
            emit(i, k, even + odd, cu);
            emit(i + 1, k, even - odd, -cu);
        }
    }
}

// Consumer warps: take the stages in order until the producer posts the end.
// GENERAL = false: every box of the launch is non-periodic and force-free, so
// only that tile body is compiled in (fewer registers than the kernel that
// carries all four bodies).
template <int ST, int SPT, bool GENERAL>
__device__ __forceinline__ void staged_consume(const SCParams& p, unsigned char* smem, StagedHeader<ST>* hd)
{
    using G = Staged<ST, SPT>;
    using E = typename Stor<ST>::E;
    for (int k = 0;; k++) {
        const int st = k % G::kStages;
        const uint32_t phase = (uint32_t)((k / G::kStages) & 1);
        const bool arrived = mbar_wait_bounded(&hd->full[st], phase, p.wait_ns);
        if (!__all_sync(0xffffffffu, arrived)) {
            // nothing arrived within the limit: flag the box, let copies still
            // in flight land (one more bounded wait) and leave
            if ((threadIdx.x & 31) == 0) {
                const int b = *reinterpret_cast<volatile const int32_t*>(&hd->t[k % (2 * G::kStages)].box);
                atomicCAS(&p.status[b >= 0 && b < p.nboxes ? b : 0], 0, LB_ERR_TIMEOUT);
            }
            mbar_wait_bounded(&hd->full[st], phase, p.wait_ns);
            return;
        }
        const StagedTile<ST>& th = hd->t[k % (2 * G::kStages)];
        const int b = th.box;
        if (b < 0) return;  // end of work
        const int64_t s0 = th.s0;
        const BoxDev& bd = th.bd;
        const unsigned char* stage = smem + kStagedHeaderBytes + st * G::kStageBytes;
        if (th.frozen) {
            // frozen box: release the stage, the state does not change
            __syncwarp();
            if ((threadIdx.x & 31) == 0) mbar_arrive(&hd->empty[st]);
            const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
            E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;
            for (int t = threadIdx.x; t < G::kSites; t += kStagedConsumers)
                if (s0 + t < bd.n3)
                    for (int i = 0; i < kQ; i++) Bb[(int64_t)i * bd.n3 + s0 + t] = Ab[(int64_t)i * bd.n3 + s0 + t];
        } else if (!GENERAL) {
            staged_tile<ST, SPT, false, false>(p, th, stage, &hd->empty[st]);
        } else if (bd.per_mask == 0) {
            if (bd.has_accel) staged_tile<ST, SPT, false, true>(p, th, stage, &hd->empty[st]);
            else staged_tile<ST, SPT, false, false>(p, th, stage, &hd->empty[st]);
        } else {
            if (bd.has_accel) staged_tile<ST, SPT, true, true>(p, th, stage, &hd->empty[st]);
            else staged_tile<ST, SPT, true, false>(p, th, stage, &hd->empty[st]);
        }
    }
}

// Producer (lane 0 of the last warp): claim tiles from the global counter
// (reset to zero by the forced re-collision at the end of every step, so a
// block that starts late -- its SM still busy with the bead kernel -- simply
// takes fewer tiles) and fill the stages as the consumers free them.
template <int ST, int SPT, bool GENERAL>
__device__ __forceinline__ void staged_produce(const SCParams& p, unsigned char* smem, StagedHeader<ST>* hd, int64_t n)
{
    using G = Staged<ST, SPT>;
    using R = typename Stor<ST>::R;
    using A = typename Stor<ST>::A;
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p.tile_counter);
    int64_t next = (int64_t)atomicAdd(ctr, 1ull);
    int last_b = -1;
    TimeWeights<R> tw{};
    int mlp_s = 0;
    for (int k = 0;; k++) {
        const int st = k % G::kStages;
        // the stage's previous tile must be released by all consumer warps; if
        // that does not happen within a second the consumers have left
        if (k >= G::kStages && !mbar_wait_bounded(&hd->empty[st], (uint32_t)(((k / G::kStages) - 1) & 1), p.wait_ns))
            return;
        const int64_t t = next;
        if (t >= p.total_tiles) {
            hd->t[k % (2 * G::kStages)].box = -1;
            mbar_arrive(&hd->full[st]);  // completes the phase with no bytes: end of work
            return;
        }
        next = (int64_t)atomicAdd(ctr, 1ull);  // the next claim overlaps this tile's copies
        const int b = locate_box(p, t);
        const BoxDev& bd = p.boxes[b];
        const int64_t s0 = (t - p.tile_prefix[b]) * G::kSites;
        if (b != last_b) {  // boundary-layer constants of this box at step n
            tw = time_weights<R>(n, bd.K, bd.time_interp, p.ring_slots);
            mlp_s = bd.mlp_row >= 0 ? mlp_substep(n, bd.K) : 0;
            last_b = b;
        }
        StagedTile<ST>& th = hd->t[k % (2 * G::kStages)];
        static_assert(sizeof(BoxDev) % 8 == 0, "box record copied in 8-byte words");
        for (int w = 0; w < (int)(sizeof(BoxDev) / 8); w++)  // word by word: few live registers
            reinterpret_cast<uint64_t*>(&th.bd)[w] = reinterpret_cast<const uint64_t*>(&bd)[w];
        if (GENERAL && bd.frame) {  // the header carries the body acceleration of step n (frame
                                    // boxes carry a body force, so they run the general kernel)
            double a[3];
            frame_accel_at(bd, p.faccel, p.ring_slots, n, a);
            for (int c = 0; c < 3; c++) th.bd.accel[c] = a[c];
        }
        th.box = b;
        th.s0 = s0;
        th.mlp_s = mlp_s;
        th.frozen = p.status[b] != 0;
        for (int a = 0; a < 4; a++) {
            th.slot[a] = tw.slot[a];
            th.c[a] = tw.c[a];
        }
        th.om = A(1) / (A)bd.tau;
        th.om1 = A(1) - th.om;
        th.srcfac = A(1) - A(0.5) * th.om;
        th.drho_b = (A)bd.rho_b - A(1);
        if (t == p.withhold_tile) {
            // test only: this stage is never armed and no copy is issued, so
            // its full barrier never completes and the consumers' bounded wait
            // runs out (the header above is in place for them to name the box)
            __threadfence_block();
            continue;
        }
        fence_proxy_async_smem();
        issue_tile<ST, SPT>(p, bd, s0, smem + kStagedHeaderBytes + st * G::kStageBytes, &hd->full[st]);
    }
}

template <int ST, int SPT, bool GENERAL>
__global__ void __launch_bounds__(kStagedThreads, 1) k_stream_collide_staged(SCParams p)
{
    using G = Staged<ST, SPT>;
    extern __shared__ __align__(128) unsigned char smem[];
    StagedHeader<ST>* hd = reinterpret_cast<StagedHeader<ST>*>(smem);
    const int64_t n = *p.step;
    if (threadIdx.x == 0) {
        for (int st = 0; st < G::kStages; st++) {
            mbar_init(&hd->full[st], 1);
            mbar_init(&hd->empty[st], kStagedConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x >= kStagedConsumers) {
        if (threadIdx.x == kStagedConsumers) staged_produce<ST, SPT, GENERAL>(p, smem, hd, n);
        return;
    }
    staged_consume<ST, SPT, GENERAL>(p, smem, hd);
}

}  // namespace lbt
