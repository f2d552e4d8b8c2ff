// blink_tables.cu -- a1/a2 (baseline uv, grid cell) and the weighting tables.
//
// One table set per channel: a coplanar, zenith-phased array has (u,v) that
// do not change with time (Sec. 4.3, Eqs. 4-5), so every time step of a
// channel shares its cells and weights.
#include "blink_common.cuh"
#include "blink_kernels.cuh"

#include <algorithm>

namespace blink {

// Antenna pair (i < j) of lexicographic baseline index b; exact integer
// result after a float estimate of the row.
__device__ __forceinline__ void pair_of(int64_t b, int n_ant, int &i, int &j) {
    const double twon1 = 2.0 * n_ant - 1.0;
    const float disc = float(twon1 * twon1 - 8.0 * double(b));
    int r = int((float(twon1) - sqrtf(fmaxf(disc, 0.f))) * 0.5f);
    r = max(0, min(r, n_ant - 2));
    auto start = [n_ant](int64_t row) { return row * (2 * int64_t(n_ant) - row - 1) / 2; };
    while (r > 0 && start(r) > b) --r;
    while (r < n_ant - 2 && start(r + 1) <= b) ++r;
    i = r;
    j = int(b - start(r)) + r + 1;
}

// One axis of a2: k = round half away from zero of (w / delta_u); false if the
// baseline leaves the grid (|k| > N/2 - 1) or is not finite.
__device__ __forceinline__ bool axis_cell(double w, double delta_u, int n_px, int &k) {
    const double t = __ddiv_rn(w, delta_u);
    if (!(fabs(t) <= 2.0 * double(n_px))) return false;
    const long long r = llround(t);
    const long long kmax = n_px / 2 - 1;
    if (r > kmax || r < -kmax) return false;
    k = int(r);
    return true;
}

// a1 + a2 for every (channel, baseline).  Grid: (ceil(B / blockDim), n_chan).
// Writes the packed canonical cell, optionally the signed cell pair, counts
// the entries of uniform-weighted channels and reduces the support bounds.
__global__ void k_cells(const double *__restrict__ ant_xyz, int n_ant, int64_t nb,
                        const ChanGeom *__restrict__ geom, ChanInfo *__restrict__ info,
                        uint32_t *__restrict__ codes, int2 *__restrict__ cells,
                        int32_t *__restrict__ counts) {
    const int ch = blockIdx.y;
    const ChanGeom g = geom[ch];
    const int64_t code_off = info[ch].code_off;
    int32_t *cnt = (counts && g.weighting == 1) ? counts + info[ch].wgt_off : nullptr;
    __shared__ double s_lambda;
    if (threadIdx.x == 0) s_lambda = __ddiv_rn(kSpeedOfLight, g.freq_hz);  // lambda = c / nu
    __syncthreads();
    const double lambda = s_lambda;
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int n = g.n_px;
    int row = -1, kabs = 0, kept = 0;
    if (b < nb) {
        int i, j;
        pair_of(b, n_ant, i, j);
        const double dx = __dsub_rn(ant_xyz[3 * j + 0], ant_xyz[3 * i + 0]);
        const double dy = __dsub_rn(ant_xyz[3 * j + 1], ant_xyz[3 * i + 1]);
        const double u = __ddiv_rn(dx, lambda);
        const double v = __ddiv_rn(dy, lambda);
        int ku = 0, kv = 0;
        uint32_t code = kCodeDropped;
        if (axis_cell(u, g.delta_u, n, ku) && axis_cell(v, g.delta_u, n, kv)) {
            // canonical half: k_v > 0, or k_v == 0 and k_u >= 0; else mirror and conjugate
            const bool mirror = kv < 0 || (kv == 0 && ku < 0);
            const int r = mirror ? -kv : kv;
            const int cu = mirror ? -ku : ku;
            const int c = cu < 0 ? cu + n : cu;
            code = pack_code(uint32_t(r), uint32_t(c), mirror ? 1u : 0u);
            row = r;
            kabs = abs(ku);
            kept = 1;
            if (cnt) atomicAdd(cnt + int64_t(r) * n + c, 1);
        } else {
            ku = kDropped;
            kv = kDropped;
        }
        codes[code_off + b] = code;
        if (cells) cells[ch * nb + b] = make_int2(ku, kv);
    }
    // warp reductions, then one atomic per warp
    const unsigned full = 0xFFFFFFFFu;
    const int wrow = __reduce_max_sync(full, row);
    const int wk = __reduce_max_sync(full, kabs);
    const unsigned wkept = __reduce_add_sync(full, unsigned(kept));
    if ((threadIdx.x & 31) == 0) {
        if (wrow >= 0) atomicMax(&info[ch].rows, wrow + 1);
        atomicMax(&info[ch].kmax_u, wk);
        atomicAdd(reinterpret_cast<unsigned long long *>(&info[ch].n_kept),
                  (unsigned long long)wkept);
    }
}

// Per channel: support rows >= 1, summed weight, and for uniform weighting
// the per-cell weight 1/n (n counts V and conj(V) entries, so the origin cell,
// whose entries all land on the canonical half, has n = 2 * count).
__global__ void k_finalize(ChanInfo *__restrict__ info, float *__restrict__ wgt) {
    const int ch = blockIdx.x;
    ChanInfo ci = info[ch];
    const int n = ci.n_px, h = n / 2;
    const int rows = max(ci.rows, 1);
    float part = 0.f;
    if (ci.weighting == 1) {
        int32_t *cnt = reinterpret_cast<int32_t *>(wgt + ci.wgt_off);
        float *w = wgt + ci.wgt_off;
        for (int64_t idx = threadIdx.x; idx < int64_t(rows) * n; idx += blockDim.x) {
            const int r = int(idx / n), c = int(idx % n);
            const int m = cnt[idx];
            float wv = 0.f;
            if (m > 0) {
                const bool origin = (r == 0 && c == 0);
                wv = __frcp_rn(float(origin ? 2 * m : m));
                // occupied cells of the full grid: the origin once, the others
                // together with their mirror
                part += origin ? 1.f : 2.f;
            }
            w[idx] = wv;
        }
    }
    // block reduction of the occupied-cell count (exact in float below 2^24)
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int k = 0; k < int(blockDim.x >> 5); ++k) tot += red[k];
        ci.rows = rows;
        ci.wsum = ci.weighting == 1 ? tot : float(2 * ci.n_kept);
        info[ch] = ci;
    }
    (void)h;
}

// Per-layer copy of the per-channel signed cells (blink_cells).
__global__ void k_expand_cells(const int2 *__restrict__ cells, const DevLayer *__restrict__ layers,
                               int n_layers, int64_t nb, int2 *__restrict__ out) {
    const int l = blockIdx.y;
    if (l >= n_layers) return;
    const DevLayer L = layers[l];
    for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < nb;
         b += int64_t(gridDim.x) * blockDim.x)
        out[int64_t(L.layer) * nb + b] = cells[int64_t(L.chan) * nb + b];
}

Error launch_tables(const double *ant_xyz, int n_ant, int64_t nb, int n_chan, const ChanGeom *geom,
                    ChanInfo *info, uint32_t *codes, int2 *cells, float *wgt, bool any_uniform,
                    cudaStream_t st) {
    if (n_chan == 0) return Error{0, ""};
    const int tpb = 256;
    dim3 grid(unsigned((nb + tpb - 1) / tpb), unsigned(n_chan));
    k_cells<<<grid, tpb, 0, st>>>(ant_xyz, n_ant, nb, geom, info, codes, cells,
                                  any_uniform ? reinterpret_cast<int32_t *>(wgt) : nullptr);
    BLINK_CUDA_TRY(cudaGetLastError());
    k_finalize<<<n_chan, 512, 0, st>>>(info, wgt);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

Error launch_expand_cells(const int2 *cells, const DevLayer *layers, int n_layers, int64_t nb,
                          int2 *out, cudaStream_t st) {
    if (n_layers == 0) return Error{0, ""};
    const int tpb = 256;
    const unsigned bx = unsigned(std::min<int64_t>((nb + tpb - 1) / tpb, 1024));
    for (int l0 = 0; l0 < n_layers; l0 += 65535) {
        const int cnt = std::min(65535, n_layers - l0);
        k_expand_cells<<<dim3(bx, unsigned(cnt)), tpb, 0, st>>>(cells, layers + l0, cnt, nb, out);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    return Error{0, ""};
}

}  // namespace blink
