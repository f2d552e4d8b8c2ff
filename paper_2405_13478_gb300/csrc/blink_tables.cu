// blink_tables.cu -- baseline uv, grid cell and the weighting tables.
//
// One table set per channel: a coplanar, zenith-phased array has (u,v) that
// do not change with time (Sec. 4.3, Eqs. 4-5), so every time step of a
// channel shares its cells and weights.
#include "blink_common.cuh"
#include "blink_div.cuh"
#include "blink_kernels.cuh"
#include "blink_pairs.cuh"

#include <algorithm>

namespace blink {

// uv and cell for every (channel, baseline).  Grid: (ceil(B / blockDim), n_chan).
// Writes the packed canonical cell, optionally the signed cell pair, counts
// the entries of uniform-weighted channels and reduces the support bounds.
__global__ void k_cells(const double *__restrict__ ant_xyz, int n_ant, int64_t nb,
                        const ChanGeom *__restrict__ geom, ChanInfo *__restrict__ info,
                        uint32_t *__restrict__ codes, int2 *__restrict__ cells,
                        int32_t *__restrict__ counts, unsigned char *__restrict__ sched,
                        unsigned char *__restrict__ csr) {
    const int ch = blockIdx.y;
    const ChanGeom g = geom[ch];
    const ChanInfo ci0 = info[ch];
    const int64_t code_off = ci0.code_off;
    int32_t *cnt = (counts && ci0.wgt_off >= 0) ? counts + ci0.wgt_off : nullptr;
    int32_t *cnt_q = nullptr, *rank = nullptr;
    if (sched && ci0.sched_off >= 0) {
        const SchedLayout lay(g.n_px, nb, ci0.n_chunks);
        cnt_q = reinterpret_cast<int32_t *>(sched + ci0.sched_off + lay.cnt_q);
        rank = reinterpret_cast<int32_t *>(sched + ci0.sched_off + lay.rank);
    }
    __shared__ double s_lambda, s_inv_lambda, s_inv_du;
    __shared__ float s_s32;
    __shared__ int32_t s_hist[kCsrMaxBuckets];  // bucket sizes of this block (row buckets)
    const bool want_csr = csr && ci0.csr_off >= 0;
    if (want_csr)
        for (int r = threadIdx.x; r < g.n_px / 2 + 1; r += blockDim.x) s_hist[r] = 0;
    if (threadIdx.x == 0) {
        s_lambda = __ddiv_rn(kSpeedOfLight, g.freq_hz);  // lambda = c / nu
        s_inv_lambda = __drcp_rn(s_lambda);
        s_inv_du = __drcp_rn(g.delta_u);
        s_s32 = float(s_inv_lambda * s_inv_du);
    }
    __syncthreads();
    const double lambda = s_lambda, inv_lambda = s_inv_lambda, inv_du = s_inv_du;
    const float s32 = s_s32;
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int n = g.n_px;
    int row = -1, kabs = 0, kept = 0;
    if (b < nb) {
        int i, j;
        baseline_pair(b, n_ant, i, j);
        const double dx = __dsub_rn(ant_xyz[3 * j + 0], ant_xyz[3 * i + 0]);
        const double dy = __dsub_rn(ant_xyz[3 * j + 1], ant_xyz[3 * i + 1]);
        int ku = 0, kv = 0;
        uint32_t code = kCodeDropped;
        if (axis_cell(dx, lambda, inv_lambda, g.delta_u, inv_du, s32, n, ku) &&
            axis_cell(dy, lambda, inv_lambda, g.delta_u, inv_du, s32, n, kv)) {
            // canonical half: k_v > 0, or k_v == 0 and k_u >= 0; else mirror and conjugate
            const bool mirror = kv < 0 || (kv == 0 && ku < 0);
            const int r = mirror ? -kv : kv;
            const int cu = mirror ? -ku : ku;
            const int c = cu < 0 ? cu + n : cu;
            code = pack_code(uint32_t(r), uint32_t(c), mirror ? 1u : 0u);
            row = r;
            kabs = abs(ku);
            kept = 1;
            const int64_t cell = int64_t(r) * n + c;
            if (cnt) atomicAdd(cnt + cell, 1);
            if (cnt_q) {
                const int q = int(b / ci0.chunk);
                rank[b] = atomicAdd(cnt_q + int64_t(q) * (n / 2) * n + cell, 1);
            }
        } else {
            ku = kDropped;
            kv = kDropped;
        }
        codes[code_off + b] = code;
        if (cells) cells[ch * nb + b] = make_int2(ku, kv);
        if (want_csr) atomicAdd(&s_hist[code == kCodeDropped ? n / 2 : int(code_row(code))], 1);
    }
    // warp reductions, a block reduction, then one atomic per block and field
    // (per-warp atomics on the channel's three fields serialised in L2)
    const unsigned full = 0xFFFFFFFFu;
    const int wrow = __reduce_max_sync(full, row);
    const int wk = __reduce_max_sync(full, kabs);
    const unsigned wkept = __reduce_add_sync(full, unsigned(kept));
    __shared__ int s_row[32], s_k[32];
    __shared__ unsigned s_kept[32];
    const int warp = int(threadIdx.x >> 5), n_warps = int((blockDim.x + 31) >> 5);
    if ((threadIdx.x & 31) == 0) {
        s_row[warp] = wrow;
        s_k[warp] = wk;
        s_kept[warp] = wkept;
    }
    __syncthreads();
    if (want_csr) {  // this block's bucket sizes (bucket-major) and the bucket totals
        const CsrLayout cl(n, nb);
        int32_t *tot = reinterpret_cast<int32_t *>(csr + ci0.csr_off + cl.tot);
        int32_t *blk = reinterpret_cast<int32_t *>(csr + ci0.csr_off + cl.blk_off);
        for (int r = threadIdx.x; r < cl.n_bkt; r += blockDim.x) {
            const int32_t c = s_hist[r];
            blk[int64_t(r) * cl.n_blk + blockIdx.x] = c;
            if (c) atomicAdd(tot + r, c);
        }
    }
    if (threadIdx.x == 0) {
        int brow = -1, bk = 0;
        unsigned long long bkept = 0;
        for (int w = 0; w < n_warps; ++w) {
            brow = max(brow, s_row[w]);
            bk = max(bk, s_k[w]);
            bkept += s_kept[w];
        }
        if (brow >= 0) atomicMax(&info[ch].rows, brow + 1);
        atomicMax(&info[ch].kmax_u, bk);
        atomicAdd(reinterpret_cast<unsigned long long *>(&info[ch].n_kept), bkept);
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

// Register-accumulation schedule, step 1 (one CTA per scheduled channel):
// rank the occupied cells by their largest per-chunk entry count and cut the
// ranking into groups of 32 (the lanes of one warp in one slot); hand the
// groups out to (slot j, warp w), heaviest group first to the warp with the
// least work so far (longest-processing-time rule); then size every (chunk,
// slot, warp) block of the entry stream to its longest lane.  A block is
// padded to the longest lane of its chunk, so cells that peak alike share a
// warp: on the 256-antenna station at 180^2 the stream holds ~1.6x the
// baselines (~2x when cells are ranked by their total count), and the
// busiest warp of a chunk -- which every chunk waits for -- carries ~5 %
// more than the mean (~30 % when groups fill the warps in rank order).
// Falls back (sched = 0) when the cells need more than kSchedSlots slots per
// thread or the padded stream outgrows its buffer, and skips channels of
// sizes <= 256 whose support rows do not fit the fused kernels.  Channels of
// larger sizes get a schedule only when flagged (sched_large) for the
// compact gridding; slot positions are r (N + 1) + c in both cases.
constexpr int kPeakBins = 64;  // peaks above 63 share the last bucket
constexpr int kMaxItems = 4096;

__global__ void __launch_bounds__(1024) k_sched_slots(ChanInfo *__restrict__ info, const float *__restrict__ wgt,
                                                      unsigned char *__restrict__ sched, int64_t nb) {
    const int ch = blockIdx.x;
    ChanInfo ci = info[ch];
    if (ci.sched_off < 0) return;
    const int n = ci.n_px, S = n + 1, R = max(ci.rows, 1), Q = ci.n_chunks;
    // channels of sizes <= 256 whose images take the two-kernel path need no
    // schedule; larger ones have one only for the compact gridding
    if (!ci.sched_large && !small_path_fits(n, R)) {
        if (threadIdx.x == 0) info[ch].sched = 0;
        return;
    }
    const SchedLayout lay(n, nb, Q);
    unsigned char *blk = sched + ci.sched_off;
    const int32_t *cnt = reinterpret_cast<const int32_t *>(wgt + ci.wgt_off);
    const int32_t *cnt_q = reinterpret_cast<const int32_t *>(blk + lay.cnt_q);
    int32_t *cell_slot = reinterpret_cast<int32_t *>(blk + lay.cell_slot);
    uint32_t *slot_pos = reinterpret_cast<uint32_t *>(blk + lay.slot_pos);
    float *slot_w = reinterpret_cast<float *>(blk + lay.slot_w);
    uint2 *meta = reinterpret_cast<uint2 *>(blk + lay.meta);
    constexpr int kWarps = 32;  // blockDim 1024
    __shared__ int whist[kWarps][kPeakBins];  // per warp and bucket: counts, then bases
    __shared__ int b_tot[kPeakBins], b_start[kPeakBins];
    __shared__ int items_l[kMaxItems], items_p[kMaxItems];
    __shared__ int g_work[kSchedSlots * kSchedWarps], g_order[kSchedSlots * kSchedWarps],
        g_place[kSchedSlots * kSchedWarps];
    __shared__ int s_occ, s_ok;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kWarps * kPeakBins; i += nt) (&whist[0][0])[i] = 0;
    __syncthreads();
    const int cells = R * n;
    const int64_t cells_all = int64_t(n / 2) * n;
    auto peak = [&](int idx) {  // largest count of the cell over the chunks
        int m = 0;
        for (int q = 0; q < Q; ++q) m = max(m, cnt_q[int64_t(q) * cells_all + idx]);
        return min(m, kPeakBins - 1);
    };
    // Deterministic ranking (the order cannot depend on thread timing, since
    // the gather's bank-aware step order follows from it): bucket by peak,
    // largest first, and by cell index inside a bucket.  Warp w ranks its
    // contiguous range of cells per bucket, 32 cells at a time (match_any
    // groups the lanes of a bucket); the bases come from the counts of the
    // lower warps and of the larger buckets.
    const int span = ((cells + kWarps - 1) / kWarps + 31) & ~31;
    const int c0 = warp * span, c1 = min(cells, c0 + span);
    for (int base = c0; base < c1; base += 32) {
        const int idx = base + lane;
        const bool occ = idx < c1 && cnt[idx] > 0;
        const int b = occ ? peak(idx) : -1;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
        const int leader = __ffs(int(peers)) - 1;
        int before = (occ && lane == leader) ? whist[warp][b] : 0;
        before = __shfl_sync(0xFFFFFFFFu, before, leader);
        if (occ) {
            cell_slot[idx] = (b << 24) | (before + __popc(peers & ((1u << lane) - 1u)));
            if (lane == leader) whist[warp][b] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    if (tid < kPeakBins) {
        int acc = 0;
        for (int w = 0; w < kWarps; ++w) {
            const int c = whist[w][tid];
            whist[w][tid] = acc;
            acc += c;
        }
        b_tot[tid] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;  // bucket starts, largest peaks first
        for (int b = kPeakBins - 1; b >= 0; --b) {
            b_start[b] = acc;
            acc += b_tot[b];
        }
        s_occ = acc;
    }
    __syncthreads();
    const int n_occ = s_occ;
    const int M = (n_occ + kSchedThreads - 1) / kSchedThreads;
    const int items = Q * max(M, 1) * kSchedWarps;
    if (M == 0 || M > kSchedSlots || items > kMaxItems) {
        if (tid == 0) {
            info[ch].sched = 0;
        }
        return;
    }
    for (int i = tid; i < kSchedSlots * kSchedThreads; i += nt) {
        slot_pos[i] = kSlotEmpty;
        slot_w[i] = 0.f;
    }
    const int G = M * kSchedWarps;  // groups of 32 ranked cells
    for (int i = tid; i < items; i += nt) items_l[i] = 0;
    __syncthreads();
    // rank of every cell (kept in cell_slot for now) and, per chunk, the
    // longest lane of every group: items_l[q G + g]
    for (int idx = c0 + lane; idx < c1; idx += 32) {
        if (cnt[idx] <= 0) continue;
        const int v = cell_slot[idx], b = v >> 24;
        const int i = b_start[b] + whist[warp][b] + (v & 0xFFFFFF);
        cell_slot[idx] = i;
        for (int q = 0; q < Q; ++q) atomicMax(&items_l[q * G + i / 32], cnt_q[int64_t(q) * cells_all + idx]);
    }
    __syncthreads();
    // groups by decreasing padded work (rank sort, ties by index) ...
    for (int g = tid; g < G; g += nt) {
        int w = 0;
        for (int q = 0; q < Q; ++q) w += items_l[q * G + g];
        g_work[g] = w;
    }
    __syncthreads();
    for (int g = tid; g < G; g += nt) {
        const int wg = g_work[g];
        int rank = 0;
        for (int h = 0; h < G; ++h) rank += g_work[h] > wg || (g_work[h] == wg && h < g);
        g_order[rank] = g;
    }
    __syncthreads();
    // ... each to the least-loaded warp that still has a free slot (lane w of
    // warp 0 tracks warp w; key = load * 32 + w, a redux.sync min per group)
    if (tid < 32) {
        const int w = tid;
        int load = 0, used = 0;
        for (int k = 0; k < G; ++k) {
            const int g = g_order[k];
            const unsigned key = (w < kSchedWarps && used < M) ? unsigned(load) * 32u + unsigned(w) : 0xFFFFFFFFu;
            const unsigned best = __reduce_min_sync(0xFFFFFFFFu, key);
            if (w == int(best & 31u)) {
                g_place[g] = used * kSchedWarps + w;  // slot j, warp w
                ++used;
                load += g_work[g];
            }
        }
    }
    __syncthreads();
    for (int idx = tid; idx < cells; idx += nt) {
        const int m = cnt[idx];
        if (m <= 0) continue;
        const int i = cell_slot[idx];
        const int jw = g_place[i / 32];
        const int j = jw / kSchedWarps, t = (jw % kSchedWarps) * 32 + i % 32;
        const int r = idx / n, c = idx % n;
        uint32_t pos = uint32_t(r * S + c);
        const bool origin = idx == 0;
        if (origin) pos |= kSlotOrigin;
        else if (r == 0) pos |= kSlotMirror;
        float w = 1.f;
        if (ci.weighting == 1) w = __frcp_rn(float(origin ? 2 * m : m));
        slot_pos[j * kSchedThreads + t] = pos;
        slot_w[j * kSchedThreads + t] = w;
        cell_slot[idx] = (j << 16) | t;
    }
    __syncthreads();
    // block lengths in stream order: group g of chunk q is block (q, slot j, warp w)
    for (int it = tid; it < items; it += nt) items_p[(it / G) * G + g_place[it % G]] = items_l[it];
    __syncthreads();
    if (tid == 0) {
        int64_t acc = 0, seg = 0, max_seg = 0;
        const int per_chunk = M * kSchedWarps;
        for (int it = 0; it < items; ++it) {
            if (it % per_chunk == 0) seg = 0;
            meta[it] = make_uint2(uint32_t(acc), uint32_t(items_p[it]));
            acc += 32 * int64_t(items_p[it]);
            seg += 32 * int64_t(items_p[it]);
            max_seg = max(max_seg, seg);
        }
        s_ok = acc <= lay.stream_cap;
        info[ch].stream_len = int32_t(acc);
        info[ch].max_seg = int32_t(max_seg);
        info[ch].m_slots = M;
        info[ch].sched = s_ok;
    }
}

// Step 2: every stream entry starts as the sentinel (index `chunk`, a zero
// staging element); step 3 then overwrites the real entries.
__global__ void k_sched_fill(const ChanInfo *__restrict__ info, unsigned char *__restrict__ sched, int64_t nb) {
    const ChanInfo ci = info[blockIdx.y];
    if (ci.sched_off < 0 || !ci.sched) return;
    const SchedLayout lay(ci.n_px, nb, ci.n_chunks);
    uint16_t *stream = reinterpret_cast<uint16_t *>(sched + ci.sched_off + lay.stream);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < ci.stream_len;
         i += int64_t(gridDim.x) * blockDim.x)
        stream[i] = uint16_t(ci.chunk);
}

// Step 3: place every kept baseline in its lane's interleaved run.
__global__ void k_sched_entries(const ChanInfo *__restrict__ info, const uint32_t *__restrict__ codes,
                                unsigned char *__restrict__ sched, int64_t nb) {
    const int ch = blockIdx.y;
    const ChanInfo ci = info[ch];
    if (ci.sched_off < 0 || !ci.sched) return;
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const uint32_t cd = codes[ci.code_off + b];
    if (cd == kCodeDropped) return;
    const int n = ci.n_px;
    const SchedLayout lay(n, nb, ci.n_chunks);
    const unsigned char *blk = sched + ci.sched_off;
    const int32_t *cell_slot = reinterpret_cast<const int32_t *>(blk + lay.cell_slot);
    const int32_t *rank = reinterpret_cast<const int32_t *>(blk + lay.rank);
    const uint2 *meta = reinterpret_cast<const uint2 *>(blk + lay.meta);
    uint16_t *stream = reinterpret_cast<uint16_t *>(sched + ci.sched_off + lay.stream);
    const int cell = int(code_row(cd)) * n + int(code_col(cd));
    const int cs = cell_slot[cell];
    const int j = cs >> 16, t = cs & 0xFFFF;
    const int q = int(b / ci.chunk);
    const uint2 m = meta[(q * ci.m_slots + j) * kSchedWarps + t / 32];
    const int64_t e = int64_t(m.x) + int64_t(rank[b]) * 32 + (t & 31);
    stream[e] = uint16_t((b - int64_t(q) * ci.chunk) | (code_conj(cd) << 15));
}

// Step 4: the atomic placement of step 3 leaves every lane's run in
// arbitrary order; fix an order that depends only on the schedule, chosen so
// that at each step the sixteen lanes of a half-warp read staged
// visibilities in distinct shared-memory bank pairs where they can (a 64-bit
// shared load of a half-warp takes one pass per distinct address sharing a
// bank pair).  On the station workload this removes about a quarter of the
// gather's bank-conflict passes.  Each lane keeps its own entries, so every
// cell still sums exactly its visibilities, in an order fixed by the
// (deterministic) schedule: images do not depend on how the plan was built.
// Blocks longer than kBankOrderMax steps are sorted by baseline index.
constexpr uint32_t kBankOrderMax = 48;

// Bank-aware order of one (chunk, slot, warp) block in shared memory, by the
// warp that owns it: lane l holds column l (stride 32); every half-warp is
// ordered on its own.  At step k each lane publishes the bank pairs of its
// remaining real entries; every lane then replays the same greedy pass over
// its half (lanes with only padding left take the sentinel; then the lanes
// that must take a real entry now, then the others, each by lane): a lane
// takes the lowest free bank pair among its own, else the sentinel if
// padding is left and its bank pair holds no real entry, else its lowest
// bank pair (a conflict).  Each lane then moves its chosen entry to step k.
// Uniform trip counts: all 32 lanes share m.
__device__ void bank_order_warp(uint16_t *col, uint32_t m, uint16_t sent, uint32_t *words, int lane) {
    const uint32_t sb = uint32_t(sent) & 15u;
    const int half = lane & 16;
    // real entries left per bank pair, 8 bits each (a block holds <= 48 entries)
    unsigned long long cnt_lo = 0, cnt_hi = 0;
    auto bump = [&](uint32_t b, long long d) {
        if (b < 8) cnt_lo += (unsigned long long)d << (8 * b);
        else cnt_hi += (unsigned long long)d << (8 * (b - 8));
    };
    uint32_t rem = 0;
    for (uint32_t j = 0; j < m; ++j) {
        const uint16_t v = col[32 * j];
        if (v != sent) {
            bump(v & 15u, 1);
            ++rem;
        }
    }
    uint32_t mask = 0;  // bank pairs with real entries left
    for (int b = 0; b < 8; ++b) {
        mask |= ((cnt_lo >> (8 * b)) & 0xFFu ? 1u : 0u) << b;
        mask |= ((cnt_hi >> (8 * b)) & 0xFFu ? 1u : 0u) << (b + 8);
    }
    for (uint32_t k = 0; k + 1 < m; ++k) {  // the last step is each lane's last entry
        words[lane] = mask;
        __syncwarp();
        const uint32_t left = m - k;
        const unsigned hm = half ? 0xFFFF0000u : 0x0000FFFFu;
        const unsigned forced_m = __ballot_sync(0xFFFFFFFFu, rem > 0 && rem == left) & hm;
        const unsigned active_m = __ballot_sync(0xFFFFFFFFu, rem > 0) & hm;
        uint32_t used = 0;
        bool sent_used = (active_m != hm);  // lanes with only padding left take the sentinel
        int mine = -1;  // -1: nothing to move, 16: the sentinel, else a bank pair
        for (int pass = 0; pass < 2; ++pass) {
            unsigned todo = pass == 0 ? forced_m : (active_m & ~forced_m);
            while (todo) {
                const int l = __ffs(int(todo)) - 1;
                todo &= todo - 1;
                const uint32_t mk = words[l] & 0xFFFFu;
                const bool forced = pass == 0;
                const uint32_t avail = mk & ~used & (sent_used ? ~(1u << sb) : 0xFFFFu);
                int ch;
                if (avail) {
                    ch = __ffs(int(avail)) - 1;
                } else if (!forced && !((used >> sb) & 1u)) {
                    ch = 16;
                } else {
                    ch = __ffs(int(mk)) - 1;
                }
                if (ch == 16) sent_used = true;
                else used |= 1u << ch;
                if (l == lane) mine = ch;
            }
        }
        __syncwarp();  // every lane has read the words before they change
        if (mine >= 0) {
            // the sentinel nearest step k, or the lowest baseline of the chosen
            // bank pair: the order depends only on the lane's set of entries
            uint32_t j = m;
            for (uint32_t i = k; i < m; ++i) {
                const uint16_t v = col[32 * i];
                if (mine == 16) {
                    if (v == sent) {
                        j = i;
                        break;
                    }
                } else if (v != sent && int(v & 15u) == mine && (j == m || (v & 0x7FFFu) < (col[32 * j] & 0x7FFFu))) {
                    j = i;
                }
            }
            const uint16_t v = col[32 * j];
            col[32 * j] = col[32 * k];
            col[32 * k] = v;
            if (mine < 16) {
                bump(uint32_t(mine), -1);
                --rem;
                const unsigned long long w = mine < 8 ? cnt_lo >> (8 * mine) : cnt_hi >> (8 * (mine - 8));
                if ((w & 0xFFu) == 0) mask &= ~(1u << mine);
            }
        }
    }
}

// 256 threads: the items of a CTA are eight whole (chunk, slot, warp)
// blocks (kSchedThreads and 256 are multiples of 32), copied to shared
// memory when at most kBankOrderMax long.
__global__ void k_sched_sort(const ChanInfo *__restrict__ info, unsigned char *__restrict__ sched,
                                                    int64_t nb) {
    const ChanInfo ci = info[blockIdx.y];
    if (ci.sched_off < 0 || !ci.sched) return;
    const SchedLayout lay(ci.n_px, nb, ci.n_chunks);
    const uint2 *meta = reinterpret_cast<const uint2 *>(sched + ci.sched_off + lay.meta);
    uint16_t *stream = reinterpret_cast<uint16_t *>(sched + ci.sched_off + lay.stream);
    const int items = ci.n_chunks * ci.m_slots * kSchedThreads;
    const uint16_t sent = uint16_t(ci.chunk);
    __shared__ uint16_t cols[8][32 * kBankOrderMax];
    __shared__ uint32_t words[8][32];
    const int wb = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    // loop bounds are CTA-uniform: every thread reaches every barrier
    for (int base = blockIdx.x * blockDim.x; base < items; base += gridDim.x * blockDim.x) {
        const int it = base + int(threadIdx.x);
        const int t = it % kSchedThreads, qj = it / kSchedThreads;
        uint2 m = make_uint2(0, 0);
        uint16_t *e = nullptr, *c = nullptr;
        if (it < items) {
            m = meta[qj * kSchedWarps + t / 32];
            e = stream + m.x + (t & 31);
            c = m.y <= kBankOrderMax ? &cols[wb][lane] : e;
            if (c != e)
                for (uint32_t a = 0; a < m.y; ++a) c[32 * a] = e[32 * a];
            // blocks short enough for the bank-aware order get it (its picks
            // depend only on each lane's set of entries); longer ones are
            // sorted by baseline index
            for (uint32_t a = 1; c == e && a < m.y; ++a) {  // insertion sort on the low 15 bits
                const uint16_t v = c[32 * a];
                uint32_t b = a;
                while (b > 0 && (c[32 * (b - 1)] & 0x7FFFu) > (v & 0x7FFFu)) {
                    c[32 * b] = c[32 * (b - 1)];
                    --b;
                }
                c[32 * b] = v;
            }
        }
        __syncwarp();
        if (it < items && c != e && m.y >= 2) bank_order_warp(c, m.y, sent, words[wb], lane);
        __syncwarp();
        if (it < items && c != e)
            for (uint32_t a = 0; a < m.y; ++a) e[32 * a] = c[32 * a];
        __syncthreads();
    }
}

// Row buckets, step 2: one warp per bucket.  The bucket's start is the sum of
// the totals of the buckets before it (row_ptr[r]; the last bucket's warp also
// writes row_ptr[n_bkt]); then an exclusive scan over the baseline blocks
// turns blk_off[r][blk] into the position of block blk's first entry of the
// bucket.  Grid: (ceil(buckets / 8), channels) x 256.
__global__ void __launch_bounds__(256) k_csr_scan(const ChanInfo *__restrict__ info, unsigned char *__restrict__ csr,
                                                  int64_t nb) {
    const ChanInfo ci = info[blockIdx.y];
    if (ci.csr_off < 0) return;
    const CsrLayout cl(ci.n_px, nb);
    const int lane = threadIdx.x & 31, r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= cl.n_bkt) return;
    const unsigned full = 0xFFFFFFFFu;
    int32_t *ptr = reinterpret_cast<int32_t *>(csr + ci.csr_off + cl.row_ptr);
    const int32_t *tot = reinterpret_cast<const int32_t *>(csr + ci.csr_off + cl.tot);
    int32_t *off = reinterpret_cast<int32_t *>(csr + ci.csr_off + cl.blk_off) + int64_t(r) * cl.n_blk;
    int32_t before = 0;
    for (int k = lane; k < r; k += 32) before += tot[k];
    before = __reduce_add_sync(full, before);
    if (lane == 0) {
        ptr[r] = before;
        if (r == cl.n_bkt - 1) ptr[r + 1] = before + tot[r];
    }
    int32_t run = before;
    for (int b0 = 0; b0 < cl.n_blk; b0 += 32) {
        const int b = b0 + lane;
        const int32_t c = b < cl.n_blk ? off[b] : 0;
        int32_t inc = c;
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t t = __shfl_up_sync(full, inc, d);
            if (lane >= d) inc += t;
        }
        if (b < cl.n_blk) off[b] = run + inc - c;
        run += __shfl_sync(full, inc, 31);
    }
}

// Row buckets, step 3: place every baseline in its bucket at its stable rank
// (earlier baselines of the same bucket first).  Blocks of kCsrBlock
// baselines, the blocks of k_cells.
__global__ void __launch_bounds__(kCsrBlock) k_csr_fill(const ChanInfo *__restrict__ info,
                                                       const uint32_t *__restrict__ codes,
                                                       unsigned char *__restrict__ csr, int64_t nb) {
    constexpr int W = kCsrBlock / 32;
    __shared__ int32_t wcnt[W][kCsrMaxBuckets];
    const ChanInfo ci = info[blockIdx.y];
    if (ci.csr_off < 0) return;
    const CsrLayout cl(ci.n_px, nb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < W * cl.n_bkt; i += kCsrBlock) wcnt[i / cl.n_bkt][i % cl.n_bkt] = 0;
    const int64_t b = int64_t(blockIdx.x) * kCsrBlock + threadIdx.x;
    uint32_t code = kCodeDropped;
    int bucket = -1;
    if (b < nb) {
        code = codes[ci.code_off + b];
        bucket = code == kCodeDropped ? ci.n_px / 2 : int(code_row(code));
    }
    const unsigned same = __match_any_sync(0xFFFFFFFFu, bucket);
    __syncthreads();
    if (bucket >= 0 && (__ffs(same) - 1) == lane) wcnt[warp][bucket] = __popc(same);
    __syncthreads();
    if (bucket < 0) return;
    int rank = __popc(same & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += wcnt[w][bucket];
    const int32_t *off = reinterpret_cast<const int32_t *>(csr + ci.csr_off + cl.blk_off);
    uint2 *ents = reinterpret_cast<uint2 *>(csr + ci.csr_off + cl.ents_by_b);
    ents[off[int64_t(bucket) * cl.n_blk + blockIdx.x] + rank] = make_uint2(uint32_t(b), code);
}

// Row buckets, step 4: inside every bucket, order the baseline-ordered
// entries by (column, baseline): up to 32 entries by a bitonic sort across the
// warp's lanes, more by a stable counting sort by column (32 entries per
// step); the dropped bucket is copied as it is.  One warp per bucket.
// Grid: (ceil(buckets / 8), channels) x 256.
__global__ void __launch_bounds__(256) k_csr_sort(const ChanInfo *__restrict__ info,
                                                  unsigned char *__restrict__ csr, int64_t nb) {
    constexpr int W = 8;
    __shared__ int32_t start[W][1024];  // per-warp column counts, then running positions
    const ChanInfo ci = info[blockIdx.y];
    if (ci.csr_off < 0) return;
    const CsrLayout cl(ci.n_px, nb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bk = blockIdx.x * W + warp;
    if (bk >= cl.n_bkt) return;
    const int32_t *ptr = reinterpret_cast<const int32_t *>(csr + ci.csr_off + cl.row_ptr);
    const uint2 *src = reinterpret_cast<const uint2 *>(csr + ci.csr_off + cl.ents_by_b);
    uint2 *dst = reinterpret_cast<uint2 *>(csr + ci.csr_off + cl.ents);
    const int p0 = ptr[bk], p1 = ptr[bk + 1];
    if (bk == cl.n_bkt - 1) {  // dropped baselines: baseline order
        for (int e = p0 + lane; e < p1; e += 32) dst[e] = src[e];
        return;
    }
    if (p1 - p0 <= 32) {
        const unsigned full = 0xFFFFFFFFu;
        const bool live = p0 + lane < p1;
        uint2 en = live ? src[p0 + lane] : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
        uint32_t kc = live ? code_col(en.y) : 0xFFFFFFFFu;  // key: (column, baseline)
        for (int k = 2; k <= 32; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint32_t okc = __shfl_xor_sync(full, kc, j);
                const uint32_t ob = __shfl_xor_sync(full, en.x, j);
                const uint32_t oc = __shfl_xor_sync(full, en.y, j);
                const bool other_less = okc < kc || (okc == kc && ob < en.x);
                const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
                if (keep_min == other_less) {
                    kc = okc;
                    en = make_uint2(ob, oc);
                }
            }
        }
        if (live) dst[p0 + lane] = en;
        return;
    }
    const int n = ci.n_px;
    int32_t *st = start[warp];
    for (int c = lane; c < n; c += 32) st[c] = 0;
    __syncwarp();
    for (int e = p0 + lane; e < p1; e += 32) atomicAdd(&st[code_col(src[e].y)], 1);
    __syncwarp();
    // exclusive scan over the n columns: lane l owns columns [l per, (l+1) per)
    const int per = (n + 31) / 32;
    int run = 0;
    for (int k = 0; k < per; ++k)
        if (lane * per + k < n) run += st[lane * per + k];
    int incl = run;
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    int acc = p0 + incl - run;
    for (int k = 0; k < per; ++k) {
        if (lane * per + k >= n) break;
        const int c = st[lane * per + k];
        st[lane * per + k] = acc;
        acc += c;
    }
    __syncwarp();
    for (int e0 = p0; e0 < p1; e0 += 32) {
        const int e = e0 + lane;
        const bool live = e < p1;
        const uint2 en = live ? src[e] : make_uint2(0u, 0u);
        const int col = live ? int(code_col(en.y)) : -1;
        const unsigned same = __match_any_sync(0xFFFFFFFFu, col);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (live) dst[st[col] + rank] = en;
        __syncwarp();
        if (live && (__ffs(same) - 1) == lane) st[col] += __popc(same);
        __syncwarp();
    }
}

// Compact gridding tables: one CTA per chunk of kCgChunk baselines of a
// channel with row buckets.  Every kept baseline of the chunk becomes the key
// cell << 12 | conj << 11 | (index in the chunk), unique inside the chunk; a
// bitonic sort in shared memory orders them by cell, then baseline (dropped
// baselines sort last as 0xFFFFFFFF).  Grid: (chunks, channels) x 256.
__global__ void __launch_bounds__(256) k_cg_sort(const ChanInfo *__restrict__ info,
                                                 const uint32_t *__restrict__ codes,
                                                 unsigned char *__restrict__ csr, int64_t nb) {
    constexpr int NT = 256;
    __shared__ uint32_t key[kCgChunk];
    __shared__ int s_cnt;
    const ChanInfo ci = info[blockIdx.y];
    // channels whose compact grid cannot fit the gridding kernel never use
    // these tables (their group cannot either)
    if (ci.csr_off < 0 || !cg_fits(max(ci.rows, 1), ci.kmax_u)) return;
    const CsrLayout cl(ci.n_px, nb);
    const int q = blockIdx.x;
    if (q >= cl.n_cg) return;
    const int64_t b0 = int64_t(q) * kCgChunk;
    const int n = int(nb - b0 < kCgChunk ? nb - b0 : int64_t(kCgChunk));
    const int N = ci.n_px, km = ci.kmax_u, kc = 2 * km + 1;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int cnt = 0;
    for (int i = threadIdx.x; i < kCgChunk; i += NT) {
        uint32_t k = 0xFFFFFFFFu;
        if (i < n) {
            const uint32_t code = codes[ci.code_off + b0 + i];
            if (code != kCodeDropped) {
                const int c = int(code_col(code)), ku = c <= N / 2 ? c : c - N;
                if (ku >= -km && ku <= km) {
                    const uint32_t cell = uint32_t(int(code_row(code)) * kc + ku + km);
                    k = (cell << 12) | (code_conj(code) << 11) | uint32_t(i);
                    ++cnt;
                }
            }
        }
        key[i] = k;
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    for (int k = 2; k <= kCgChunk; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < kCgChunk / 2; t += NT) {
                const int i = 2 * t - (t & (j - 1)), l = i + j;  // i has bit j clear
                const uint32_t x = key[i], y = key[l];
                if ((x > y) == ((i & k) == 0)) {
                    key[i] = y;
                    key[l] = x;
                }
            }
            __syncthreads();
        }
    }
    uint32_t *dst = reinterpret_cast<uint32_t *>(csr + ci.csr_off + cl.cg_ents) + int64_t(q) * kCgChunk;
    for (int i = threadIdx.x; i < kCgChunk; i += NT) dst[i] = key[i];
    if (threadIdx.x == 0) reinterpret_cast<int32_t *>(csr + ci.csr_off + cl.cg_cnt)[q] = s_cnt;
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

// Summed weight of every layer of a group (used where the image kernels do
// not write it themselves).
__global__ void k_wsum(const DevLayer *__restrict__ layers, int n_layers, const ChanInfo *__restrict__ chans,
                       float *__restrict__ wsum) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < n_layers) wsum[layers[l].layer] = chans[layers[l].chan].wsum;
}

Error launch_wsum_copy(const ImageArgs &a, cudaStream_t st) {
    if (!a.wsum_out || a.n_layers == 0) return Error{0, ""};
    k_wsum<<<(a.n_layers + 255) / 256, 256, 0, st>>>(a.layers, a.n_layers, a.chans, a.wsum_out);
    BLINK_CUDA_TRY(cudaGetLastError());
    return Error{0, ""};
}

Error launch_tables(const double *ant_xyz, int n_ant, int64_t nb, int n_chan, const ChanGeom *geom,
                    ChanInfo *info, uint32_t *codes, int2 *cells, float *wgt, bool any_counts,
                    cudaStream_t st, unsigned char *sched, unsigned char *csr) {
    if (n_chan == 0) return Error{0, ""};
    const int tpb = kCsrBlock;  // k_cells' blocks are the blocks of the row-bucket sort
    dim3 grid(unsigned((nb + tpb - 1) / tpb), unsigned(n_chan));
    k_cells<<<grid, tpb, 0, st>>>(ant_xyz, n_ant, nb, geom, info, codes, cells,
                                  any_counts ? reinterpret_cast<int32_t *>(wgt) : nullptr, sched, csr);
    BLINK_CUDA_TRY(cudaGetLastError());
    if (sched) {
        k_sched_slots<<<n_chan, 1024, 0, st>>>(info, wgt, sched, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_sched_fill<<<dim3(64, unsigned(n_chan)), 256, 0, st>>>(info, sched, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_sched_entries<<<grid, tpb, 0, st>>>(info, codes, sched, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
        // one CTA per 256 items of the largest possible schedule: every block
        // is ordered by its own warp in one pass (blocks beyond a channel's
        // schedule return at once)
        const int64_t q_max = (nb + kSchedMaxChunk - 1) / kSchedMaxChunk;
        const unsigned sort_ctas = unsigned((q_max * kSchedSlots * kSchedThreads + 255) / 256);
        k_sched_sort<<<dim3(sort_ctas, unsigned(n_chan)), 256, 0, st>>>(info, sched, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
    if (csr) {
        k_csr_scan<<<dim3(unsigned((kCsrMaxBuckets + 7) / 8), unsigned(n_chan)), 256, 0, st>>>(info, csr, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_csr_fill<<<dim3(unsigned((nb + kCsrBlock - 1) / kCsrBlock), unsigned(n_chan)), kCsrBlock, 0, st>>>(
            info, codes, csr, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_csr_sort<<<dim3(unsigned((kCsrMaxBuckets + 7) / 8), unsigned(n_chan)), 256, 0, st>>>(info, csr, nb);
        BLINK_CUDA_TRY(cudaGetLastError());
        k_cg_sort<<<dim3(unsigned((nb + kCgChunk - 1) / kCgChunk), unsigned(n_chan)), 256, 0, st>>>(info, codes, csr,
                                                                                                  nb);
        BLINK_CUDA_TRY(cudaGetLastError());
    }
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
