// Synthetic coarse flow: the random-phase Kolmogorov-spectrum field that
// stands in for the DNS velocity record sampled around a tracer (Sec. 2-3):
//
//   u(x, t) = sum_m amp_m cos(kvec_m . (x - xc) + omega_m t + phi_m).
//
// Evaluated in FP64 with separable phase factors: exp(i kvec_ma (x_a - xc))
// is tabulated per axis, the time factor exp(i (omega_m t + phi_m)) per block
// in shared memory, and each site multiplies three or four unit complex
// numbers per mode instead of calling cos.  Also the per-box conservation
// finaliser (FP64 partial sums added in a fixed order).
#include <cstdio>

#include "lbt_kernels.cuh"

namespace lbt {

constexpr int kSynthThreads = 256;
constexpr int kSynthMaxModes = 3072;  // time factors of all modes fit 48 KB of shared memory

// T[a][m][x] = exp(i kvec[m][a] (x - xc)), a = 0..2, x = 0..X-1 (X >= E: a
// zoomed coarse grid may reach past the box), xc = (E - 1)/2.
__global__ void k_synth_axis(const double* kvec, int M, int E, int X, double2* T)
{
    const double xc = 0.5 * (E - 1);
    const int64_t total = 3LL * M * X;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % X);
        const int m = (int)((t / X) % M);
        const int a = (int)(t / ((int64_t)X * M));
        double s, c;
        sincos(kvec[3 * m + a] * (x - xc), &s, &c);
        T[t] = make_double2(c, s);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One block per (sample, face, chunk of face points).  The points are the
// coarse face grid: every z-th site, Ec = (E - 1)/z + 1 per side (every site
// when z = 1).  out[j][f][c][Q][P].
template <class R>
__global__ void __launch_bounds__(kSynthThreads) k_synth_faces(const double2* T, const double* amp, const double* omega,
                                                              const double* phi, int M, int E, int X, int z, int K,
                                                              int64_t j0, int chunks_per_face, R* out)
{
    const int Ec = coarse_points(E, z);
    extern __shared__ double2 sC[];  // exp(i (omega t + phi)) * T[fixed axis][m][fixed coordinate]
    const int chunk = blockIdx.x % chunks_per_face;
    const int f = (blockIdx.x / chunks_per_face) % 6;
    const int64_t j = blockIdx.x / (chunks_per_face * 6);
    const double t = (double)((j0 + j) * K);
    const int fa = f / 2;
    const int fx = (f & 1) ? E - 1 : 0;
    const int ap = fa == 0 ? 1 : 0;
    const int aq = fa == 2 ? 1 : 2;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double s, c;
        sincos(omega[m] * t + phi[m], &s, &c);
        sC[m] = cmul(make_double2(c, s), T[((int64_t)fa * M + m) * X + fx]);
    }
    __syncthreads();
    const int64_t fe = (int64_t)Ec * Ec;
    const int64_t per_chunk = (fe + chunks_per_face - 1) / chunks_per_face;
    const int64_t s0 = chunk * per_chunk;
    const int64_t s1 = min(fe, s0 + per_chunk);
    for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        const int p = (int)(s % Ec) * z, q = (int)(s / Ec) * z;
        double u0 = 0, u1 = 0, u2 = 0;
        for (int m = 0; m < M; m++) {
            const double2 zp = T[((int64_t)ap * M + m) * X + p];
            const double2 zq = T[((int64_t)aq * M + m) * X + q];
            const double2 w = cmul(sC[m], zp);
            const double re = w.x * zq.x - w.y * zq.y;
            u0 += amp[3 * m] * re;
            u1 += amp[3 * m + 1] * re;
            u2 += amp[3 * m + 2] * re;
        }
        R* o = out + (j * 6 + f) * 3 * fe;
        o[s] = (R)u0;
        o[fe + s] = (R)u1;
        o[2 * fe + s] = (R)u2;
    }
}

// Field on the coarse grid (every zm-th site, Ec = (E - 1)/zm + 1 per axis):
// out[c][Z][Y][X].
template <class R>
__global__ void __launch_bounds__(kSynthThreads) k_synth_volume(const double2* T, const double* amp, const double* omega,
                                                               const double* phi, int M, int E, int X, int zm, double t,
                                                               R* out)
{
    const int Ec = coarse_points(E, zm);
    extern __shared__ double2 sC[];
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        double s, c;
        sincos(omega[m] * t + phi[m], &s, &c);
        sC[m] = make_double2(c, s);
    }
    __syncthreads();
    const int64_t n3 = (int64_t)Ec * Ec * Ec;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n3; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % Ec) * zm, y = (int)((s / Ec) % Ec) * zm, z = (int)(s / ((int64_t)Ec * Ec)) * zm;
        double u0 = 0, u1 = 0, u2 = 0;
        for (int m = 0; m < M; m++) {
            const double2 w = cmul(cmul(sC[m], T[(int64_t)m * X + x]), T[((int64_t)M + m) * X + y]);
            const double2 zz = T[((int64_t)2 * M + m) * X + z];
            const double re = w.x * zz.x - w.y * zz.y;
            u0 += amp[3 * m] * re;
            u1 += amp[3 * m + 1] * re;
            u2 += amp[3 * m + 2] * re;
        }
        out[s] = (R)u0;
        out[n3 + s] = (R)u1;
        out[2 * n3 + s] = (R)u2;
    }
}

static int grid_for_synth(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

cudaError_t launch_synth_faces(const double* kvec, const double* amp, const double* omega, const double* phi,
                               int M, int E, int zoom, int K, int64_t j0, int64_t nsamp, int out_f64, void* out,
                               void* workspace, cudaStream_t s)
{
    if (M > kSynthMaxModes) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    double2* T = reinterpret_cast<double2*>(workspace);
    const int Ec = coarse_points(E, zoom);
    const int X = (Ec - 1) * zoom + 1 > E ? (Ec - 1) * zoom + 1 : E;  // <= 2E - 1: fits the workspace
    k_synth_axis<<<grid_for_synth(3LL * M * X), 256, 0, s>>>(kvec, M, E, X, T);
    const int64_t fe = (int64_t)Ec * Ec;
    const int chunks = (int)((fe + 1023) / 1024);
    const size_t smem = sizeof(double2) * M;
    for (int64_t j = 0; j < nsamp; j += 4096) {
        const int64_t nj = min((int64_t)4096, nsamp - j);
        const unsigned grid = (unsigned)(nj * 6 * chunks);
        if (out_f64)
            k_synth_faces<double><<<grid, kSynthThreads, smem, s>>>(T, amp, omega, phi, M, E, X, zoom, K, j0 + j, chunks,
                                                                   reinterpret_cast<double*>(out) + j * 6 * 3 * fe);
        else
            k_synth_faces<float><<<grid, kSynthThreads, smem, s>>>(T, amp, omega, phi, M, E, X, zoom, K, j0 + j, chunks,
                                                                  reinterpret_cast<float*>(out) + j * 6 * 3 * fe);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_synth_volume(const double* kvec, const double* amp, const double* omega, const double* phi,
                                int M, int E, int zoom, double t, int out_f64, void* out, void* workspace,
                                cudaStream_t s)
{
    if (M > kSynthMaxModes) return cudaErrorInvalidValue;
    double2* T = reinterpret_cast<double2*>(workspace);
    const int Ec = coarse_points(E, zoom);
    const int X = (Ec - 1) * zoom + 1 > E ? (Ec - 1) * zoom + 1 : E;
    k_synth_axis<<<grid_for_synth(3LL * M * X), 256, 0, s>>>(kvec, M, E, X, T);
    const int64_t n3 = (int64_t)Ec * Ec * Ec;
    const size_t smem = sizeof(double2) * M;
    const int grid = (int)min((int64_t)152 * 8, (n3 + kSynthThreads - 1) / kSynthThreads);
    if (out_f64)
        k_synth_volume<double><<<grid, kSynthThreads, smem, s>>>(T, amp, omega, phi, M, E, X, zoom, t,
                                                                 reinterpret_cast<double*>(out));
    else
        k_synth_volume<float><<<grid, kSynthThreads, smem, s>>>(T, amp, omega, phi, M, E, X, zoom, t,
                                                                reinterpret_cast<float*>(out));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Vorticity diagnostic: |curl u| by central differences over the cube
// [lo, hi]^3 of a box's velocity field u [3][E^3] (real type R), FP64 sums.
// Each block writes the sum of its sites (grid-stride order, then a fixed
// tree); one thread adds the block sums in order and divides by the count.
constexpr int kVortThreads = 256;
constexpr int kVortMaxBlocks = 512;

template <class R>
__global__ void __launch_bounds__(kVortThreads) k_vort_partial(const R* u, int E, int lo, int hi, double* partial)
{
    const int m = hi - lo + 1;
    const int64_t cube = (int64_t)m * m * m, n3 = (int64_t)E * E * E;
    const int64_t sy = E, sz = (int64_t)E * E;
    const R* ux = u;
    const R* uy = u + n3;
    const R* uz = u + 2 * n3;
    double acc = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cube; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = lo + (int)(s % m), y = lo + (int)((s / m) % m), z = lo + (int)(s / ((int64_t)m * m));
        const int64_t c = (int64_t)z * sz + (int64_t)y * sy + x;
        const double wx = 0.5 * ((double)uz[c + sy] - (double)uz[c - sy]) - 0.5 * ((double)uy[c + sz] - (double)uy[c - sz]);
        const double wy = 0.5 * ((double)ux[c + sz] - (double)ux[c - sz]) - 0.5 * ((double)uz[c + 1] - (double)uz[c - 1]);
        const double wz = 0.5 * ((double)uy[c + 1] - (double)uy[c - 1]) - 0.5 * ((double)ux[c + sy] - (double)ux[c - sy]);
        acc += sqrt(wx * wx + wy * wy + wz * wz);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[kVortThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void k_vort_final(const double* partial, int nblocks, double count, double* out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; b++) t += partial[b];
    out[0] = t / count;
}

cudaError_t launch_vorticity(const void* u, int u_f64, int E, int lo, int hi, double* scratch, double* out,
                             cudaStream_t s)
{
    const int64_t m = hi - lo + 1, cube = m * m * m;
    int64_t g = (cube + kVortThreads - 1) / kVortThreads;
    if (g > kVortMaxBlocks) g = kVortMaxBlocks;
    if (u_f64)
        k_vort_partial<double><<<(unsigned)g, kVortThreads, 0, s>>>(reinterpret_cast<const double*>(u), E, lo, hi,
                                                                    scratch);
    else
        k_vort_partial<float><<<(unsigned)g, kVortThreads, 0, s>>>(reinterpret_cast<const float*>(u), E, lo, hi,
                                                                   scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_vort_final<<<1, 32, 0, s>>>(scratch, (int)g, (double)cube, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_cons_final(const BoxDev* boxes, const ChainDev* chains, int nboxes, int64_t chunks,
                             const double* partial, const double* vel, double* out, int32_t* status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nboxes) return;
    const BoxDev& bd = boxes[b];
    const int64_t nch = (bd.n3 + kConsChunk - 1) / kConsChunk;
    double t[4] = {0, 0, 0, 0};
    for (int64_t c = 0; c < nch && c < chunks; c++)
        for (int a = 0; a < 4; a++) t[a] += partial[((int64_t)b * chunks + c) * 4 + a];
    double pb[3] = {0, 0, 0};
    if (bd.chain >= 0) {
        const ChainDev& ch = chains[bd.chain];
        for (int i = 0; i < ch.nbeads; i++)
            for (int a = 0; a < 3; a++) pb[a] += vel[3 * (ch.bead_off + i) + a];
        for (int a = 0; a < 3; a++) pb[a] *= ch.mass;
    }
    double* o = out + 8 * (int64_t)b;
    o[0] = (double)bd.n3 + t[0];
    for (int a = 0; a < 3; a++) {
        o[1 + a] = t[1 + a];
        o[4 + a] = pb[a];
    }
    o[7] = 0.0;
    bool finite = isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2]) && isfinite(t[3]);
    if (!finite || !(o[0] > 0.0)) atomicCAS(&status[b], 0, LB_ERR_NONFINITE);
}

}  // namespace lbt

int lbt_staged_tile_sites(int spt) { return lbt::staged_tile_sites(spt); }
bool lbt_staged_spt_ok(int storage, int spt) { return lbt::staged_spt_ok(storage, spt); }
int lbt_staged_default_spt(int storage) { return lbt::staged_default_spt(storage); }
