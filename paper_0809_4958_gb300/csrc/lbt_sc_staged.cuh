// Stream-collide with the boundary layer, staged through shared memory by
// TMA bulk copies (cp.async.bulk) in a two-stage pipeline.
//
// A tile is kStageSites consecutive sites of one box (4 KB of one population
// row).  For population i the sites of a tile pull from one contiguous
// source range shifted by c_iy E + c_iz E^2 (and by c_ix inside the row), so
// one bulk copy per population, widened by a 16-byte halo on each side for
// the x shift, brings everything the tile needs into shared memory; the x
// shift becomes an offset into that row.  Each persistent block keeps the
// copies for its next tile in flight while it computes the current one, so
// DRAM sees a steady stream instead of load-compute-store bursts.
//
// Only sites whose pull source crosses a periodic face (a wrap) read global
// memory directly.  Copies are clamped to the box's arrays; sites whose
// source lies outside are boundary sites, which are overwritten with the
// boundary equilibrium anyway.
#pragma once
#include "lbt_device.cuh"

namespace lbt {

constexpr int kStagedThreads = 512;
constexpr int kStagedHaloBytes = 16;                           // x-shift halo on each side

// Tile geometry: two stages of 4 KB rows.  (Four stages of 2 KB rows measured
// slower on GB300: the cost per bulk copy and per tile grows faster than the
// gain from the deeper pipeline.)
template <int ST>
struct Staged {
    using E = typename Stor<ST>::E;
    static constexpr int kRowBytes = 4096;                                  // one population row of a tile
    static constexpr int kStages = 2;
    static constexpr int kRowStride = kRowBytes + 2 * kStagedHaloBytes;
    static constexpr int kStageBytes = kQ * kRowStride;
    static constexpr int kSmemBytes = kStages * kStageBytes + 64;          // + mbarriers
    static constexpr int kSites = kRowBytes / (int)sizeof(E);              // sites per tile
    static constexpr int kSPT = kSites / kStagedThreads;                   // sites per thread
    static constexpr int kHalo = kStagedHaloBytes / (int)sizeof(E);        // halo elements
    static_assert(kSPT >= 1, "tile smaller than the block");
};

// Sites per tile of the staged kernel (host side, for the tile table).
inline int staged_tile_sites(int storage)
{
    return storage == kF64 ? Staged<kF64>::kSites
                           : (storage == kF32 ? Staged<kF32>::kSites : Staged<kF16>::kSites);
}

// ---- PTX helpers (mbarrier + bulk copy) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase of the barrier, giving up after about one second.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase)
{
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase))
        if (global_ns() - t0 > 1000000000ull) return false;
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

// Producer (one thread): bulk copies of the 19 source rows of a tile.
template <int ST>
__device__ __forceinline__ void issue_tile(const SCParams& p, int64_t tile, unsigned char* stage, uint64_t* bar)
{
    using E = typename Stor<ST>::E;
    constexpr int T = Staged<ST>::kSites, H = Staged<ST>::kHalo;
    const int b = locate_box(p, tile);
    const BoxDev& bd = p.boxes[b];
    const int64_t n3 = bd.n3, Ei = bd.E;
    const int64_t s0 = (tile - p.tile_prefix[b]) * T;
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
        bulk_load(stage + i * Staged<ST>::kRowStride + (lo[i] - start) * sizeof(E), Ab + (int64_t)i * n3 + lo[i],
                  (uint32_t)((hi[i] - lo[i]) * sizeof(E)), bar);
    }
}

// Quotient and remainder of a site index by E with a precomputed multiplier:
// q = (s * m) >> 40 with m = ceil(2^40 / E), exact for s < 2^31 and E <= 1024.
__device__ __forceinline__ int div_e(int64_t s, uint64_t m) { return (int)(((uint64_t)s * m) >> 40); }

// Consumer: thread t collides sites t, t + kStagedThreads, ... of the tile,
// so the lanes of a warp read consecutive shared-memory words (no bank
// conflicts) and store consecutive global words.
template <int ST, bool PER, bool ACCEL>
__device__ __forceinline__ void staged_tile(const SCParams& p, const BoxDev& bd, int64_t s0, int64_t n,
                                            const unsigned char* stage)
{
    using S = Stor<ST>;
    using E = typename S::E;
    using A = typename S::A;
    using R = typename S::R;
    constexpr int SPT = Staged<ST>::kSPT, H = Staged<ST>::kHalo;

    const int Ei = bd.E;
    const int64_t n3 = bd.n3;
    const uint64_t mE = bd.div_magic;
    const int per = bd.per_mask;
    const bool px = per & 1, py = per & 2, pz = per & 4;
    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;

    int xs_[SPT], ys_[SPT], zs_[SPT];
    bool act[SPT], bnd[SPT];
    bool any_bnd = false;
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        const int64_t s = s0 + threadIdx.x + k * kStagedThreads;
        act[k] = s < n3;
        const int64_t sc = act[k] ? s : 0;
        const int row = div_e(sc, mE);
        const int x = (int)(sc - (int64_t)row * Ei);
        const int z = div_e(row, mE);
        const int y = row - z * Ei;
        xs_[k] = x;
        ys_[k] = y;
        zs_[k] = z;
        bnd[k] = act[k] && ((!px && (x == 0 || x == Ei - 1)) || (!py && (y == 0 || y == Ei - 1)) ||
                            (!pz && (z == 0 || z == Ei - 1)));
        any_bnd |= bnd[k];
    }

    // f_i pulled into site k: shared memory, or global memory across a periodic wrap
    auto fval = [&](int i, int k) -> A {
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        if (PER) {
            const int xs = xs_[k] - cx, ys = ys_[k] - cy, zs = zs_[k] - cz;
            const bool wrap = (px && (xs < 0 || xs >= Ei)) || (py && (ys < 0 || ys >= Ei)) ||
                              (pz && (zs < 0 || zs >= Ei));
            if (wrap)
                return S::in(Ab[(int64_t)i * n3 +
                                ((int64_t)wrapi(zs, Ei) * Ei + wrapi(ys, Ei)) * Ei + wrapi(xs, Ei)]);
        }
        const E* row = reinterpret_cast<const E*>(stage + i * Staged<ST>::kRowStride);
        return S::in(row[H + threadIdx.x + k * kStagedThreads - cx]);
    };

    A drho[SPT], ux[SPT], uy[SPT], uz[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        A r = A(0), jx = A(0), jy = A(0), jz = A(0);
        if (act[k] && !bnd[k]) {
#pragma unroll
            for (int i = 0; i < kQ; i++) {
                const A f = fval(i, k);
                r += f;
                if (cvec(i, 0)) jx += cvec(i, 0) * f;
                if (cvec(i, 1)) jy += cvec(i, 1) * f;
                if (cvec(i, 2)) jz += cvec(i, 2) * f;
            }
        }
        const A rho = A(1) + r;
        const A inv = A(1) / rho;
        if (ACCEL) {
            jx += A(0.5) * rho * (A)bd.accel[0];
            jy += A(0.5) * rho * (A)bd.accel[1];
            jz += A(0.5) * rho * (A)bd.accel[2];
        }
        drho[k] = r;
        ux[k] = jx * inv;
        uy[k] = jy * inv;
        uz[k] = jz * inv;
    }
    if (any_bnd) {
        const TimeWeights<R> tw = time_weights<R>(n, bd.K, bd.time_interp, p.ring_slots);
        const R* ring = reinterpret_cast<const R*>(p.ring);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            if (bnd[k]) {
                int pp, qq;
                const int f = owning_face(xs_[k], ys_[k], zs_[k], Ei, per, pp, qq);
                R ub[3];
                boundary_velocity<R>(ring, p.ring_slot_elems, bd.ring_off, Ei, f, pp, qq, tw, ub);
                add_mlp_residual<R>(p, bd, n, f, pp, qq, ub);
                drho[k] = (A)bd.rho_b - A(1);
                ux[k] = (A)ub[0];
                uy[k] = (A)ub[1];
                uz[k] = (A)ub[2];
            }
        }
    }
    const A om = A(1) / (A)bd.tau;
    const A srcfac = A(1) - A(0.5) * om;
    A usq[SPT], ua[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        usq[k] = A(1.5) * (ux[k] * ux[k] + uy[k] * uy[k] + uz[k] * uz[k]);
        if (ACCEL) ua[k] = ux[k] * (A)bd.accel[0] + uy[k] * (A)bd.accel[1] + uz[k] * (A)bd.accel[2];
    }
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const A w = wgt<A>(i);
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            const A rho = A(1) + drho[k];
            A cu = A(0);
            if (cx) cu += cx * ux[k];
            if (cy) cu += cy * uy[k];
            if (cz) cu += cz * uz[k];
            const A deq = w * (drho[k] + rho * (A(3) * cu + A(4.5) * cu * cu - usq[k]));
            A val = deq;
            if (!bnd[k]) {
                const A f = fval(i, k);
                val = f + om * (deq - f);
                if (ACCEL) {
                    const A ca = (A)(cx * bd.accel[0] + cy * bd.accel[1] + cz * bd.accel[2]);
                    val += srcfac * w * rho * (A(3) * (ca - ua[k]) + A(9) * cu * ca);
                }
            }
            if (act[k]) Bb[(int64_t)i * n3 + s0 + threadIdx.x + k * kStagedThreads] = S::out(val);
        }
    }
}

// Persistent blocks take tiles from a global counter (reset to zero by the
// forced re-collision at the end of every step), so a block that starts late
// -- its SM still busy with the bead kernel -- simply takes fewer tiles.
template <int ST>
__global__ void __launch_bounds__(kStagedThreads, 1) k_stream_collide_staged(SCParams p)
{
    constexpr int kStagedStages = Staged<ST>::kStages;
    constexpr int kStagedStageBytes = Staged<ST>::kStageBytes;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStagedStages * kStagedStageBytes);
    __shared__ int64_t sTile[kStagedStages];
    constexpr int T = Staged<ST>::kSites;
    const int64_t n = *p.step;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStagedStages; st++) mbar_init(&bar[st], 1);
        fence_mbar_init();
        for (int st = 0; st < kStagedStages; st++) {
            const int64_t t = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(p.tile_counter), 1ull);
            sTile[st] = t < p.total_tiles ? t : -1;
            if (t < p.total_tiles) issue_tile<ST>(p, t, smem + st * kStagedStageBytes, &bar[st]);
        }
    }
    __syncthreads();
    for (int k = 0;; k++) {
        const int st = k % kStagedStages;
        const int64_t tile = sTile[st];
        if (tile < 0) break;  // later fetches are larger: nothing else is in flight
        const uint32_t phase = (uint32_t)((k / kStagedStages) & 1);
        const int b = locate_box(p, tile);
        const BoxDev& bd = p.boxes[b];
        const bool arrived = mbar_wait_bounded(&bar[st], phase);
        if (!__syncthreads_and(arrived)) {
            // the copies did not arrive within a second: flag the box, give the
            // copies one more bounded wait, and leave (the whole block at once)
            if (threadIdx.x == 0) atomicCAS(&p.status[b], 0, LB_ERR_TIMEOUT);
            mbar_wait_bounded(&bar[st], phase);
            return;
        }
        const int64_t s0 = (tile - p.tile_prefix[b]) * T;
        const unsigned char* stage = smem + st * kStagedStageBytes;
        if (p.status[b] != 0) {
            // frozen box: the state does not change
            using E = typename Stor<ST>::E;
            const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
            E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;
            for (int t = threadIdx.x; t < T; t += blockDim.x)
                if (s0 + t < bd.n3)
                    for (int i = 0; i < kQ; i++) Bb[(int64_t)i * bd.n3 + s0 + t] = Ab[(int64_t)i * bd.n3 + s0 + t];
        } else if (bd.per_mask == 0) {
            if (bd.has_accel) staged_tile<ST, false, true>(p, bd, s0, n, stage);
            else staged_tile<ST, false, false>(p, bd, s0, n, stage);
        } else {
            if (bd.has_accel) staged_tile<ST, true, true>(p, bd, s0, n, stage);
            else staged_tile<ST, true, false>(p, bd, s0, n, stage);
        }
        __syncthreads();  // every thread is done with this stage
        if (threadIdx.x == 0) {
            const int64_t t = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(p.tile_counter), 1ull);
            sTile[st] = t < p.total_tiles ? t : -1;
            if (t < p.total_tiles) {
                fence_proxy_async_smem();
                issue_tile<ST>(p, t, smem + st * kStagedStageBytes, &bar[st]);
            }
        }
    }
}

}  // namespace lbt
