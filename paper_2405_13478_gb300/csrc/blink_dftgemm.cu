// blink_dftgemm.cu -- pass 2 of the image transform as a dense GEMM on the
// fifth-generation tensor cores (tcgen05), in BF16 or FP16 with FP32
// accumulation and optional split-precision recovery.
//
// After pass 1 (gridding + inverse DFT of every canonical row along u, the
// same kernel as the FFT path) a layer holds T[k][p], k < R (support rows),
// p the FFT-order column.  The real image is
//   I[y][x] = sum_{k<R} c_k (cos(2 pi k y'/N) Re T[k][p] - sin(2 pi k y'/N) Im T[k][p])
// with y' = y - N/2, x = (p + N/2) mod N, c_0 = 1 and c_k = 2 (Hermitian
// symmetry along v; Sec. 4.3 Eq. 6, Sec. 5.2.2).  That is I = A B with
//   A[y][k] = c_k cos(..) for k < Rp, -c_{k-Rp} sin(..) for Rp <= k < 2 Rp,
//   B[k][p] = Re T[k][p] (k < Rp), Im T[k - Rp][p] (Rp <= k < 2 Rp),
// a real GEMM of M = N, N = N, K = 2 Rp (Rp = R rounded up to 8).  A depends
// only on (N, Rp) and is built once in FP64 with exact integer phase
// reduction; B is converted per layer.
//
// Precision: x = hi + lo with hi = round(x) and lo = round((x - hi) 2^s) 2^-s;
// the split product keeps A_hi B_hi + A_hi B_lo + A_lo B_hi (the A_lo B_lo
// term is below FP32 resolution).  FP16 needs range control: every layer's B
// is scaled by a power of two so its largest entry is below 2^14, and the
// cross terms (lo scaled by 2^11) go to a second TMEM accumulator.
//
// Operands sit in shared memory in the K-major core-matrix layout of the
// tensor cores (8 rows x 16 bytes per core matrix, no swizzle); global memory
// holds them already in that layout so each tile arrives with one 1-D TMA
// bulk copy.  One CTA computes one 128-row output tile, 256 columns wide for
// a single product and 128 wide for the split modes (two CTAs per SM): 4
// warps, thread 0 issues the MMAs, TMEM holds the FP32 accumulators, and
// tcgen05.ld reads them back for the epilogue, which transposes each warp's
// 32 x 32 block through shared memory so every image store covers 128
// contiguous bytes of a row.  Every wait is bounded; a timeout sets the
// status word and the CTA still releases its tensor memory.
#include "blink_common.cuh"
#include "blink_kernels.cuh"
#include "blink_sync.cuh"
#include "blink_grid_sorted.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace blink {

namespace {

constexpr int kTileM = 128, kTileN = 256;
// Output columns of a pass-2 tile: 256 for one product; 128 for the split
// modes, whose four operand tiles then take 96 KB of shared memory (K = 96)
// so two CTAs share an SM (and their TMEM accumulators fit its 512 columns).
template <int SPLIT>
constexpr int tile_n() { return SPLIT == 3 ? 128 : kTileN; }

struct DftArgs {
    const uint16_t *a_hi, *a_lo;  // [N / 128] blocks of 128 x K (tiled)
    const uint16_t *b_hi, *b_lo;  // [layers][N / 256] blocks of 256 x K (tiled)
    const int *b_exp;             // per-layer power-of-two scale of B (FP16)
    const DevLayer *layers;
    const ChanInfo *chans;
    float *out;
    uint32_t flags;
    int n_px, K;
    int *status;
    const float *ref;             // reference images (fused epilogue) or null
    unsigned long long wait_ns;   // limit of the first barrier waits (failure tests lower it)
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Element (r, k) of a tile with K columns in the K-major core-matrix layout.
__host__ __device__ __forceinline__ int tiled(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((addr >> 4) & 0x3FFF);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;  // descriptor version of this tensor-core generation; no swizzle
    return d;
}

template <bool FP16>
__device__ __forceinline__ uint16_t to_bits(float x) {
    if constexpr (FP16) {
        return __half_as_ushort(__float2half_rn(x));
    } else {
        return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    }
}
template <bool FP16>
__device__ __forceinline__ float from_bits(uint16_t b) {
    if constexpr (FP16) {
        return __half2float(__ushort_as_half(b));
    } else {
        return __bfloat162float(__ushort_as_bfloat16(b));
    }
}

template <bool FP16>
constexpr int lo_shift() { return FP16 ? 11 : 0; }

// ---------------------------------------------------------------- operand A
// A[y][k] for one image size, hi and lo parts, tiled per 128-row block.
template <bool FP16>
__global__ void k_dft_table(int N, int Rp, uint16_t *a_hi, uint16_t *a_lo) {
    const int K = 2 * Rp;
    const int64_t total = int64_t(N) * K;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int y = int(i / K), k = int(i % K);
        const int kk = k < Rp ? k : k - Rp;
        const int64_t m = ((int64_t(kk) * (y - N / 2)) % N + N) % N;  // exact phase index
        double s, c;
        sincospi(2.0 * double(m) / double(N), &s, &c);
        const double ck = kk == 0 ? 1.0 : 2.0;
        const float x = float(k < Rp ? ck * c : -ck * s);
        const uint16_t hb = to_bits<FP16>(x);
        const float lo = (x - from_bits<FP16>(hb)) * float(1 << lo_shift<FP16>());
        const int64_t o = int64_t(y / kTileM) * kTileM * K + tiled(y % kTileM, k, K);
        a_hi[o] = hb;
        a_lo[o] = to_bits<FP16>(lo);
    }
}

// ---------------------------------------------------------------- operand B
// Per layer: T (FP32 complex [r_alloc][N] in scratch) -> B hi/lo tiles.
// One CTA per layer.  FP16: scale 2^-e with the largest |entry| below 2^14.
template <bool FP16, int SPLIT>
__global__ void __launch_bounds__(256) k_split(const float2 *__restrict__ T, int r_alloc, int N, int Rp,
                                               const DevLayer *__restrict__ layers,
                                               const ChanInfo *__restrict__ chans, int l0, uint16_t *b_hi,
                                               uint16_t *b_lo, int *b_exp) {
    const int lw = blockIdx.x;
    const DevLayer L = layers[l0 + lw];
    const int R = chans[L.chan].rows;
    const int K = 2 * Rp;
    const float2 *t = T + int64_t(lw) * r_alloc * N;
    float scale = 1.f;
    if constexpr (FP16) {
        float m = 0.f;
        for (int i = threadIdx.x; i < R * N; i += blockDim.x) m = fmaxf(m, fmaxf(fabsf(t[i].x), fabsf(t[i].y)));
        __shared__ float red[256];
        red[threadIdx.x] = m;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (int(threadIdx.x) < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        int e = 0;
        if (red[0] > 0.f) e = max(ilogbf(red[0]) - 13, -100);
        if (threadIdx.x == 0) b_exp[lw] = e;
        scale = ldexpf(1.f, -e);
    }
    uint16_t *hi = b_hi + int64_t(lw) * N * K;
    uint16_t *lo = b_lo + int64_t(lw) * N * K;
    const float lo_scale = float(1 << lo_shift<FP16>());
    // one thread per (column p, group of 8 k): 16-byte stores
    for (int i = threadIdx.x; i < N * (K / 8); i += blockDim.x) {
        const int p = i % N, k8 = i / N;
        uint16_t h[8], l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * k8 + j;
            const int r = k < Rp ? k : k - Rp;
            float x = 0.f;
            if (r < R) x = (k < Rp ? t[int64_t(r) * N + p].x : t[int64_t(r) * N + p].y) * scale;
            h[j] = to_bits<FP16>(x);
            l[j] = to_bits<FP16>((x - from_bits<FP16>(h[j])) * lo_scale);
        }
        constexpr int TN = tile_n<SPLIT>();
        const int64_t o = int64_t(p / TN) * TN * K + tiled(p % TN, 8 * k8, K);
        uint4 hv, lv;
        hv.x = h[0] | (uint32_t(h[1]) << 16); hv.y = h[2] | (uint32_t(h[3]) << 16);
        hv.z = h[4] | (uint32_t(h[5]) << 16); hv.w = h[6] | (uint32_t(h[7]) << 16);
        lv.x = l[0] | (uint32_t(l[1]) << 16); lv.y = l[2] | (uint32_t(l[3]) << 16);
        lv.z = l[4] | (uint32_t(l[5]) << 16); lv.w = l[6] | (uint32_t(l[7]) << 16);
        *reinterpret_cast<uint4 *>(hi + o) = hv;
        *reinterpret_cast<uint4 *>(lo + o) = lv;
    }
}

// ----------------------------------------------------------------- the GEMM
template <int NC>
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Grid: (N / 128, N / 256, layers of the wave).  128 threads.
template <bool FP16, int SPLIT>
__global__ void __launch_bounds__(128, SPLIT == 3 ? 2 : 1) k_dftgemm(DftArgs d, int l0, float *__restrict__ out,
                                                    const float *__restrict__ ref) {
    constexpr bool CROSS = FP16 && SPLIT == 3;      // separate accumulator for the cross terms
    constexpr int TN = tile_n<SPLIT>();
    constexpr uint32_t NCOL = CROSS ? 2 * TN : TN;   // TMEM columns
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    const int K = d.K, N = d.n_px, H = N / 2;
    const int mt = blockIdx.x, nt = blockIdx.y, lw = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_bytes = uint32_t(kTileM) * K * 2, b_bytes = uint32_t(TN) * K * 2;
    unsigned char *sA_hi = smem_tc, *sA_lo = smem_tc + a_bytes;
    unsigned char *sB_hi = smem_tc + (SPLIT == 3 ? 2 : 1) * a_bytes;
    unsigned char *sB_lo = sB_hi + b_bytes;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar_load)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint32_t total = (SPLIT == 3 ? 2 : 1) * (a_bytes + b_bytes);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&bar_load)), "r"(total)
                     : "memory");
        const int n_tiles = N / TN;
        const uint16_t *ga[2] = {d.a_hi + int64_t(mt) * kTileM * K, d.a_lo + int64_t(mt) * kTileM * K};
        const int64_t bo = (int64_t(lw) * n_tiles + nt) * TN * K;
        const uint16_t *gb[2] = {d.b_hi + bo, d.b_lo + bo};
        unsigned char *sa[2] = {sA_hi, sA_lo}, *sb[2] = {sB_hi, sB_lo};
        for (int h = 0; h < (SPLIT == 3 ? 2 : 1); ++h) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    saddr(sa[h])),
                "l"(ga[h]), "r"(a_bytes), "r"(saddr(&bar_load))
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    saddr(sb[h])),
                "l"(gb[h]), "r"(b_bytes), "r"(saddr(&bar_load))
                : "memory");
        }
    }
    // every decision below is CTA-uniform (the epilogue's tcgen05.ld is
    // warp-collective, and the MMAs are issued only if all threads agree)
    const bool loaded = __syncthreads_and(wait_parity(saddr(&bar_load), 0, d.wait_ns));
    bool ok = loaded;
    if (tid == 0 && loaded) {
        // D = A B^T over K in steps of 16: M = 128, N = 256, both K-major
        constexpr uint32_t fmt = FP16 ? 0u : 1u;  // 0 FP16, 1 BF16
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(TN >> 3) << 17) |
                               (uint32_t(kTileM >> 4) << 24);
        const uint32_t sbo = uint32_t(K / 8) * 128;
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ah = smem_desc(saddr(sA_hi) + s * 256, 128, sbo);
            const uint64_t bh = smem_desc(saddr(sB_hi) + s * 256, 128, sbo);
            mma_f16(tmem, ah, bh, idesc, s > 0);
            if constexpr (SPLIT == 3) {
                const uint64_t al = smem_desc(saddr(sA_lo) + s * 256, 128, sbo);
                const uint64_t bl = smem_desc(saddr(sB_lo) + s * 256, 128, sbo);
                const uint32_t tx = CROSS ? tmem + TN : tmem;
                mma_f16(tx, ah, bl, idesc, CROSS ? uint32_t(s > 0) : 1u);
                mma_f16(tx, al, bh, idesc, 1u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr(&bar_mma))
                     : "memory");
    }
    if (loaded) ok = __syncthreads_and(wait_parity(saddr(&bar_mma), 0, d.wait_ns));
    if (!ok) {
        if (tid == 0 && d.status) atomicExch(d.status, -4);  // BLINK_ERR_TIMEOUT
        // let copies or MMAs still in flight finish before the memory goes away
        wait_parity(saddr(&bar_load), 0);
        if (loaded) wait_parity(saddr(&bar_mma), 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const DevLayer L = d.layers[l0 + lw];
        const ChanInfo ci = d.chans[L.chan];
        float scale = ((d.flags & 1u) && ci.wsum > 0.f) ? 1.f / ci.wsum : 1.f;
        if (FP16) scale = ldexpf(scale, d.b_exp[lw]);
        const float cross = 1.f / float(1 << lo_shift<FP16>());
        // the operands are consumed: each warp transposes its 32 x 32 blocks
        // through shared memory, so every store instruction writes one image
        // row's 32 consecutive columns (128 bytes) instead of 32 rows' pieces
        float *stg = reinterpret_cast<float *>(smem_tc) + warp * (32 * 33);
        float *img = out + L.out_off;
        const float *rimg = ref ? ref + L.out_off : nullptr;
        const int y0 = mt * kTileM + warp * 32;
        for (int c0 = 0; c0 < TN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32<32>(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
            uint32_t q[32];
            if constexpr (CROSS) tmem_ld32<32>(tmem + (uint32_t(warp * 32) << 16) + uint32_t(TN + c0), q);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float e = __uint_as_float(r[j]);
                if constexpr (CROSS) e = fmaf(__uint_as_float(q[j]), cross, e);
                stg[lane * 33 + j] = e * scale;
            }
            __syncwarp();
            const int x = (nt * TN + c0 + H) % N + lane;  // 32 contiguous image columns
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                const int64_t o = int64_t(y0 + i) * N + x;
                float v = stg[i * 33 + lane];
                if (rimg) v -= __ldcs(rimg + o);  // fused epilogue: dirty - reference
                __stcs(img + o, v);
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

// ------------------------------------------------- pass 1 as a GEMM (BF16)
// When the gridded support is narrow (|k_u| <= kmax), pass 1 is also a dense
// real GEMM over the compact columns c = -kmax..kmax (Kc of them, padded to 8):
//   T[r][p] = sum_c G[r][c] exp(+2 pi i c p / N)   (r < R, p FFT-order column),
//   [Tr | Ti] (R x 2N) = [Gr | Gi] (R x 2Kc) B1^T  with, for n = (part, p),
//   B1[(0, p)][k] = cos th (k < Kc), -sin th (k >= Kc);
//   B1[(1, p)][k] = sin th (k < Kc),  cos th (k >= Kc),   th = 2 pi c_k p / N,
// c_k = (k mod Kc) - kmax.  k_grid_a1 grids a layer straight into the compact
// A1 = [Gr | Gi] (hi/lo, tiled, 128 rows), k_gemm1 multiplies on the tensor
// cores and writes T in the layout of the pass-2 operand B (hi/lo), so the FP32
// row FFT and the split pass are not needed.  BF16 only (no range control).
constexpr int kTile1N = 128;  // output columns of one pass-1 CTA

__global__ void k_row_table(int N, int kmax, int Kc, uint16_t *b_hi, uint16_t *b_lo) {
    const int K1 = 2 * Kc;
    const int64_t total = int64_t(2 * N) * K1;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int n = int(i / K1), k = int(i % K1);
        const int part = n / N, p = n % N, kk = k % Kc;
        float x = 0.f;
        if (kk <= 2 * kmax) {
            const int64_t m = ((int64_t(kk - kmax) * p) % N + N) % N;  // exact phase index
            double sn, cs;
            sincospi(2.0 * double(m) / double(N), &sn, &cs);
            const bool re_in = k < Kc;
            x = float(part == 0 ? (re_in ? cs : -sn) : (re_in ? sn : cs));
        }
        const uint16_t hb = to_bits<false>(x);
        const int64_t o = int64_t(n / kTile1N) * kTile1N * K1 + tiled(n % kTile1N, k, K1);
        b_hi[o] = hb;
        b_lo[o] = to_bits<false>(x - from_bits<false>(hb));
    }
}

struct Grid1Args {
    const float2 *vis;
    const DevLayer *layers;
    const ChanInfo *chans;
    const uint32_t *codes;
    const float *wgt;
    const unsigned char *csr;
    int64_t nb;
    int n_px, kmax, Kc;
    uint16_t *a_hi, *a_lo;  // [wave] blocks of 128 x 2 Kc (tiled)
    const float2 *cg;       // compact grids of the wave's layers (k_grid_compact), or null
    int64_t cg_stride;
};

// Grid: (bands of 8 rows, layers of the wave).  Compact gridding of rows
// [8 band, 8 band + 8) of one layer (columns |k_u| <= kmax), weights,
// Hermitian completion of row 0, then those rows of A1 (hi/lo).  With two
// layers per A1 block (support <= 64 rows) layer lw fills rows 64 (lw & 1) +.
__global__ void __launch_bounds__(256) k_grid_a1(Grid1Args g, int l0, int pack) {
    extern __shared__ float2 gc[];  // [8][Kc]
    const int band = blockIdx.x, lw = blockIdx.y;
    const DevLayer L = g.layers[l0 + lw];
    const ChanInfo ci = g.chans[L.chan];
    const int R = ci.rows, Kc = g.Kc, kmax = g.kmax, N = g.n_px, H = N / 2, K1 = 2 * Kc;
    const int r0 = band * 8;
    // bands past the layer's support still write their (zero) rows: the A1
    // block may hold a larger-support layer of an earlier wave
    const int nrows = max(0, min(8, R - r0));
    const int tid = threadIdx.x, nt = blockDim.x;
    auto zero = [&]() {
        for (int i = tid; i < 8 * Kc; i += nt) gc[i] = make_float2(0.f, 0.f);
    };
    const float2 *vis = g.vis + L.vis_off;
    if (g.cg) {
        // the layer's compact grid, already weighted and complete: copy the
        // band's rows (its columns |k_u| <= kmax of the channel)
        const int km = ci.kmax_u, kc = 2 * km + 1;
        const float2 *src = g.cg + int64_t(lw) * g.cg_stride + int64_t(r0) * kc;
        zero();
        __syncthreads();
        for (int i = tid; i < nrows * kc; i += nt) {
            const int r = i / kc, c = i % kc;
            gc[r * Kc + (c - km + kmax)] = __ldcs(src + i);
        }
    } else if (nrows == 0) {
        // nothing to grid: the rows below are written as zeros
        zero();
        __syncthreads();
    } else if (g.csr && ci.csr_off >= 0) {
        // only this band's baselines, from the sorted row buckets: the same
        // deterministic, atomic-free sums as the FP32 path
        const CsrLayout cl(N, g.nb);
        auto cell = [&](uint32_t key) -> float2 * {
            const int col = int(key & 0xFFFFu), ku = col <= H ? col : col - N;
            return (ku < -kmax || ku > kmax) ? nullptr : gc + int(key >> 16) * Kc + (ku + kmax);
        };
        grid_band_sorted<256>(r0, nrows, reinterpret_cast<const int32_t *>(g.csr + ci.csr_off + cl.row_ptr),
                              reinterpret_cast<const uint2 *>(g.csr + ci.csr_off + cl.ents), vis,
                              LayerGains{nullptr, nullptr, 0}, tid, cell, zero);
    } else {
        // a channel without row buckets: shared-memory atomics over the code table
        zero();
        __syncthreads();
        const uint32_t *code = g.codes + ci.code_off;
        for (int64_t b = tid; b < g.nb; b += nt) {
            const uint32_t cd = __ldg(code + b);
            if (cd == kCodeDropped) continue;
            const int r = int(code_row(cd)) - r0, col = int(code_col(cd));
            const int ku = col <= H ? col : col - N;
            if (r < 0 || r >= nrows || ku < -kmax || ku > kmax) continue;
            float2 v = __ldcs(vis + b);
            if (code_conj(cd)) v.y = -v.y;
            float2 *cell = gc + r * Kc + (ku + kmax);
            atomicAdd(&cell->x, v.x);
            atomicAdd(&cell->y, v.y);
        }
    }
    __syncthreads();
    const float *w = ci.weighting == 1 && !g.cg ? g.wgt + ci.wgt_off : nullptr;
    if (w)
        for (int i = tid; i < nrows * Kc; i += nt) {
            const int r = i / Kc, kk = i % Kc, ku = kk - kmax;
            if (r0 + r == 0 || kk > 2 * kmax) continue;
            const float wv = w[(r0 + r) * N + (ku < 0 ? ku + N : ku)];
            gc[i].x *= wv;
            gc[i].y *= wv;
        }
    __syncthreads();
    // row 0: k_u >= 0 was gridded; weight it and mirror the conjugate to -k_u;
    // the origin carries V and conj V of its baselines: 2 Re * w
    if (r0 == 0 && !g.cg)
        for (int ku = tid; ku <= kmax; ku += nt) {
            const float wv = w ? w[ku] : 1.f;
            const float2 v = gc[kmax + ku];
            if (ku == 0) {
                gc[kmax] = make_float2(2.f * v.x * wv, 0.f);
            } else {
                gc[kmax + ku] = make_float2(v.x * wv, v.y * wv);
                gc[kmax - ku] = make_float2(v.x * wv, -v.y * wv);
            }
        }
    __syncthreads();
    // A1 rows: k < Kc real parts, k >= Kc imaginary parts (rows >= R of the band zero)
    const int blk = pack ? lw >> 1 : lw, roff = pack ? 64 * (lw & 1) : 0;
    uint16_t *hi = g.a_hi + int64_t(blk) * 128 * K1;
    uint16_t *lo = g.a_lo + int64_t(blk) * 128 * K1;
    for (int i = tid; i < 8 * (K1 / 8); i += nt) {
        const int r = i % 8, k8 = i / 8;
        uint16_t h[8], l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * k8 + j, kk = k % Kc;
            float x = 0.f;
            if (r < nrows) x = k < Kc ? gc[r * Kc + kk].x : gc[r * Kc + kk].y;
            h[j] = to_bits<false>(x);
            l[j] = to_bits<false>(x - from_bits<false>(h[j]));
        }
        const int o = tiled(roff + r0 + r, 8 * k8, K1);
        uint4 hv, lv;
        hv.x = h[0] | (uint32_t(h[1]) << 16); hv.y = h[2] | (uint32_t(h[3]) << 16);
        hv.z = h[4] | (uint32_t(h[5]) << 16); hv.w = h[6] | (uint32_t(h[7]) << 16);
        lv.x = l[0] | (uint32_t(l[1]) << 16); lv.y = l[2] | (uint32_t(l[3]) << 16);
        lv.z = l[4] | (uint32_t(l[5]) << 16); lv.w = l[6] | (uint32_t(l[7]) << 16);
        *reinterpret_cast<uint4 *>(hi + o) = hv;
        *reinterpret_cast<uint4 *>(lo + o) = lv;
    }
}

struct Gemm1Args {
    const uint16_t *a_hi, *a_lo;  // [wave] 128 x K1 (tiled)
    const uint16_t *b_hi, *b_lo;  // B1 table, [2N / 128] blocks of 128 x K1
    uint16_t *t_hi, *t_lo;        // pass-2 operand B: [wave][N / 256] blocks of 256 x K2
    const DevLayer *layers;
    const ChanInfo *chans;
    int n_px, K1, Rp;
    int *status;
    unsigned long long wait_ns;
};

// Grid: (2N / 128, A1 blocks of the wave).  128 threads; D (128 x 128, FP32
// in TMEM) = A1 B1^T over K1, then each row r < Rp of a layer (TMEM lane r, or
// 64 + r for the second layer of a packed block) goes to column k2 = r (real
// part) or Rp + r (imaginary part) of that layer's pass-2 operand.
template <int SPLIT>
__global__ void __launch_bounds__(128, 1) k_gemm1(Gemm1Args d, int l0, int pack, int cnt) {
    constexpr uint32_t NCOL = kTile1N;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    const int K1 = d.K1, N = d.n_px, Rp = d.Rp, K2 = 2 * Rp;
    const int nt = blockIdx.x, blk = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_bytes = 128u * K1 * 2, b_bytes = uint32_t(kTile1N) * K1 * 2;
    unsigned char *sA_hi = smem_tc, *sA_lo = smem_tc + a_bytes;
    unsigned char *sB_hi = smem_tc + (SPLIT == 3 ? 2 : 1) * a_bytes;
    unsigned char *sB_lo = sB_hi + b_bytes;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar_load)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint32_t total = (SPLIT == 3 ? 2 : 1) * (a_bytes + b_bytes);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&bar_load)), "r"(total)
                     : "memory");
        const uint16_t *ga[2] = {d.a_hi + int64_t(blk) * 128 * K1, d.a_lo + int64_t(blk) * 128 * K1};
        const uint16_t *gb[2] = {d.b_hi + int64_t(nt) * kTile1N * K1, d.b_lo + int64_t(nt) * kTile1N * K1};
        unsigned char *sa[2] = {sA_hi, sA_lo}, *sb[2] = {sB_hi, sB_lo};
        for (int h = 0; h < (SPLIT == 3 ? 2 : 1); ++h) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    saddr(sa[h])),
                "l"(ga[h]), "r"(a_bytes), "r"(saddr(&bar_load))
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    saddr(sb[h])),
                "l"(gb[h]), "r"(b_bytes), "r"(saddr(&bar_load))
                : "memory");
        }
    }
    const bool loaded = __syncthreads_and(wait_parity(saddr(&bar_load), 0, d.wait_ns));
    bool ok = loaded;
    if (tid == 0 && loaded) {
        // D = A1 B1^T over K1 in steps of 16: M = 128, N = 128, both K-major, BF16
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kTile1N >> 3) << 17) |
                               (uint32_t(128 >> 4) << 24);
        const uint32_t sbo = uint32_t(K1 / 8) * 128;
        for (int s = 0; s < K1 / 16; ++s) {
            const uint64_t ah = smem_desc(saddr(sA_hi) + s * 256, 128, sbo);
            const uint64_t bh = smem_desc(saddr(sB_hi) + s * 256, 128, sbo);
            mma_f16(tmem, ah, bh, idesc, s > 0);
            if constexpr (SPLIT == 3) {
                const uint64_t al = smem_desc(saddr(sA_lo) + s * 256, 128, sbo);
                const uint64_t bl = smem_desc(saddr(sB_lo) + s * 256, 128, sbo);
                mma_f16(tmem, ah, bl, idesc, 1u);
                mma_f16(tmem, al, bh, idesc, 1u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr(&bar_mma))
                     : "memory");
    }
    if (loaded) ok = __syncthreads_and(wait_parity(saddr(&bar_mma), 0, d.wait_ns));
    if (!ok) {
        if (tid == 0 && d.status) atomicExch(d.status, -4);  // BLINK_ERR_TIMEOUT
        wait_parity(saddr(&bar_load), 0);
        if (loaded) wait_parity(saddr(&bar_mma), 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = warp * 32 + lane;  // TMEM lane = row of D
        const int lw = pack ? 2 * blk + (row >> 6) : blk, r = pack ? row & 63 : row;
        const bool live = lw < cnt;
        const int R = live ? d.chans[d.layers[l0 + lw].chan].rows : 0;
        uint16_t *th = d.t_hi + int64_t(lw) * N * K2;
        uint16_t *tl = d.t_lo + int64_t(lw) * N * K2;
        for (int c0 = 0; c0 < kTile1N; c0 += 32) {
            uint32_t v[32];
            tmem_ld32<32>(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (live && r < Rp) {
                const int n0 = nt * kTile1N + c0;  // 32 columns of one part (N % 128 == 0)
                const int part = n0 / N, k2 = part ? Rp + r : r;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int p = (n0 + j) % N;
                    const float x = r < R ? __uint_as_float(v[j]) : 0.f;
                    const uint16_t hb = to_bits<false>(x);
                    constexpr int TN = tile_n<SPLIT>();
                    const int64_t o = int64_t(p / TN) * TN * K2 + tiled(p % TN, k2, K2);
                    th[o] = hb;
                    tl[o] = to_bits<false>(x - from_bits<false>(hb));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

template <bool FP16, int SPLIT>
Error run_mode(int N, const ImageArgs &a, int Rp, cudaStream_t st) {
    const int K = 2 * Rp;
    const size_t a_elems = size_t(N) * K;
    const size_t t_bytes = size_t(a.r_alloc) * N * sizeof(float2);
    const size_t b_elems = size_t(N) * K;
    const size_t per_layer = t_bytes + 2 * b_elems * 2 + 16;
    const size_t fixed = 2 * a_elems * 2 + 256;
    if (!a.scratch || a.scratch_bytes < fixed + per_layer)
        return Error{-5, "tensor-core transform scratch too small"};
    const int wave = int(std::min<size_t>(size_t(a.n_layers), std::min<size_t>(65535, (a.scratch_bytes - fixed) / per_layer)));
    unsigned char *base = reinterpret_cast<unsigned char *>(a.scratch);
    uint16_t *a_hi = reinterpret_cast<uint16_t *>(base);
    uint16_t *a_lo = a_hi + a_elems;
    unsigned char *wave_base = base + ((fixed + 255) / 256) * 256;
    float2 *T = reinterpret_cast<float2 *>(wave_base);
    uint16_t *b_hi = reinterpret_cast<uint16_t *>(wave_base + size_t(wave) * t_bytes);
    uint16_t *b_lo = b_hi + size_t(wave) * b_elems;
    int *b_exp = reinterpret_cast<int *>(b_lo + size_t(wave) * b_elems);
    constexpr int TN = tile_n<SPLIT>();
    const size_t smem = size_t(SPLIT == 3 ? 2 : 1) * (size_t(kTileM) + TN) * K * 2;
    // both passes on the tensor cores when the compact support fits (BF16)
    const int Kc = (2 * a.kmax + 1 + 7) / 8 * 8, K1 = 2 * Kc;
    const size_t smem1 = size_t(SPLIT == 3 ? 2 : 1) * (128 + kTile1N) * size_t(K1) * 2;
    if (!FP16 && !a.gains && a.kmax > 0 && a.r_alloc <= 128 && smem1 <= 227 * 1024) {
        const size_t b1_elems = size_t(2 * N) * K1, a1_elems = size_t(128) * K1;
        const size_t fixed1 = 2 * a_elems * 2 + 2 * b1_elems * 2 + 512;
        const size_t per1 = 2 * a1_elems * 2 + 2 * b_elems * 2;
        if (a.scratch_bytes < fixed1 + per1) return Error{-5, "tensor-core transform scratch too small"};
        int wave1 = int(std::min<size_t>(size_t(a.n_layers), std::min<size_t>(65535, (a.scratch_bytes - fixed1) / per1)));
        if (a.cg) wave1 = std::min(wave1, a.cg_cap);
        uint16_t *b1_hi = a_lo + a_elems, *b1_lo = b1_hi + b1_elems;
        unsigned char *wb = base + ((fixed1 + 255) / 256) * 256;
        uint16_t *a1_hi = reinterpret_cast<uint16_t *>(wb), *a1_lo = a1_hi + size_t(wave1) * a1_elems;
        uint16_t *t_hi = a1_lo + size_t(wave1) * a1_elems, *t_lo = t_hi + size_t(wave1) * b_elems;
        k_dft_table<false><<<256, 256, 0, st>>>(N, Rp, a_hi, a_lo);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_row_table<<<256, 256, 0, st>>>(N, a.kmax, Kc, b1_hi, b1_lo);
        BLINK_CUDA_TRY(cudaGetLastError());
        const size_t smem_g = size_t(8) * Kc * sizeof(float2);
        const int pack = a.r_alloc <= 64 ? 1 : 0;  // two layers per 128-row A1 block
        // rows of A1 no band writes (>= R of a layer, the unused half of a pair) stay zero
        BLINK_CUDA_TRY(cudaMemsetAsync(a1_hi, 0, 2 * size_t(wave1) * a1_elems * sizeof(uint16_t), st));
        BLINK_CUDA_TRY(cudaFuncSetAttribute(k_gemm1<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem1)));
        BLINK_CUDA_TRY(cudaFuncSetAttribute(k_dftgemm<FP16, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        const unsigned long long wns = a.wait_ns < 0 ? kWaitNs : static_cast<unsigned long long>(a.wait_ns);
        for (int l0 = 0; l0 < a.n_layers; l0 += wave1) {
            const int cnt = std::min(wave1, a.n_layers - l0);
            if (pack && (cnt & 1)) {  // odd wave: the last block's second half must read zero
                BLINK_CUDA_TRY(cudaMemsetAsync(a1_hi + size_t(cnt / 2) * a1_elems, 0, a1_elems * sizeof(uint16_t), st));
                BLINK_CUDA_TRY(cudaMemsetAsync(a1_lo + size_t(cnt / 2) * a1_elems, 0, a1_elems * sizeof(uint16_t), st));
            }
            if (a.cg) {
                Error e = launch_grid_compact(a, l0, cnt, st);
                if (e.status) return e;
            }
            Grid1Args g1{a.vis, a.layers, a.chans, a.codes, a.wgt, a.csr, a.nb, N, a.kmax, Kc, a1_hi, a1_lo,
                         a.cg, a.cg_stride};
            k_grid_a1<<<dim3(unsigned((a.r_alloc + 7) / 8), unsigned(cnt)), 256, smem_g, st>>>(g1, l0, pack);
            BLINK_CUDA_TRY(cudaGetLastError());
            Gemm1Args d1{a1_hi, a1_lo, b1_hi, b1_lo, t_hi, t_lo, a.layers, a.chans, N, K1, Rp, a.status, wns};
            const int blocks = pack ? (cnt + 1) / 2 : cnt;
            k_gemm1<SPLIT><<<dim3(unsigned(2 * N / kTile1N), unsigned(blocks)), 128, smem1, st>>>(d1, l0, pack, cnt);
            BLINK_CUDA_TRY(cudaGetLastError());
            DftArgs d{a_hi, a_lo, t_hi, t_lo, nullptr, a.layers, a.chans, static_cast<float *>(a.out), a.flags, N, K,
                      a.status, a.ref, wns};
            k_dftgemm<FP16, SPLIT><<<dim3(unsigned(N / kTileM), unsigned(N / TN), unsigned(cnt)), 128, smem, st>>>(
                d, l0, d.out, d.ref);
            BLINK_CUDA_TRY(cudaGetLastError());
        }
        return Error{0, ""};
    }
    k_dft_table<FP16><<<256, 256, 0, st>>>(N, Rp, a_hi, a_lo);
    BLINK_CUDA_TRY(cudaGetLastError());
    BLINK_CUDA_TRY(cudaFuncSetAttribute(k_dftgemm<FP16, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    const int wave_r = a.cg ? std::min(wave, a.cg_cap) : wave;
    for (int l0 = 0; l0 < a.n_layers; l0 += wave_r) {
        const int cnt = std::min(wave_r, a.n_layers - l0);
        ImageArgs ra = a;
        ra.scratch = T;
        ra.scratch_bytes = size_t(wave) * t_bytes;
        if (ra.cg) {
            Error e = launch_grid_compact(ra, l0, cnt, st);
            if (e.status) return e;
            ra.cg_l0 = l0;
        }
        Error e = launch_rows_wave(N, ra, l0, cnt, st);
        if (e.status) return e;
        k_split<FP16, SPLIT><<<cnt, 256, 0, st>>>(T, a.r_alloc, N, Rp, a.layers, a.chans, l0, b_hi, b_lo, b_exp);
        BLINK_CUDA_TRY(cudaGetLastError());
        DftArgs d{a_hi, a_lo, b_hi, b_lo, b_exp, a.layers, a.chans, static_cast<float *>(a.out), a.flags, N, K, a.status,
                  a.ref, a.wait_ns < 0 ? kWaitNs : static_cast<unsigned long long>(a.wait_ns)};
        k_dftgemm<FP16, SPLIT><<<dim3(unsigned(N / kTileM), unsigned(N / TN), unsigned(cnt)), 128, smem, st>>>(
            d, l0, d.out, d.ref);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

}  // namespace

bool dftgemm_supported(int n_px, int r_alloc, int mode) {
    const int Rp = (r_alloc + 7) / 8 * 8;
    const bool split = mode == 2 || mode == 4;
    const size_t smem = size_t(split ? 2 : 1) * (size_t(kTileM) + (split ? tile_n<3>() : tile_n<1>())) * 2 * Rp * 2;
    return n_px >= kTileN && n_px % kTileN == 0 && image_size_supported(n_px) && 2 * Rp <= 256 &&
           smem <= 227 * 1024;
}

size_t dftgemm_scratch_fixed(int n_px, int r_alloc, int kmax) {
    const int Rp = (r_alloc + 7) / 8 * 8;
    const int K1 = 2 * ((2 * kmax + 1 + 7) / 8 * 8);
    return 2 * size_t(n_px) * 2 * Rp * 2 + 2 * size_t(2 * n_px) * K1 * 2 + 1024;
}

size_t dftgemm_scratch_per_layer(int n_px, int r_alloc) {
    const int Rp = (r_alloc + 7) / 8 * 8;
    return size_t(r_alloc) * n_px * sizeof(float2) + 2 * size_t(n_px) * 2 * Rp * 2 + 16;
}

Error launch_dftgemm_group(int n_px, int mode, const ImageArgs &a, cudaStream_t st) {
    if (a.n_layers == 0) return Error{0, ""};
    if (!dftgemm_supported(n_px, a.r_alloc, mode)) return Error{-2, "tensor-core transform: unsupported size or support"};
    const int Rp = (a.r_alloc + 7) / 8 * 8;
    const bool split = mode == 2 || mode == 4;
    const size_t smem = size_t(split ? 2 : 1) * (size_t(kTileM) + (split ? tile_n<3>() : tile_n<1>())) * 2 * Rp * 2;
    if (2 * Rp > 256 || smem > 227 * 1024)
        return Error{-2, "tensor-core transform: too many support rows for shared memory"};
    switch (mode) {
        case 1: return run_mode<false, 1>(n_px, a, Rp, st);
        case 2: return run_mode<false, 3>(n_px, a, Rp, st);
        case 3: return run_mode<true, 1>(n_px, a, Rp, st);
        case 4: return run_mode<true, 3>(n_px, a, Rp, st);
        default: return Error{-1, "unknown transform mode"};
    }
}

}  // namespace blink
