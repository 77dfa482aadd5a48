// rv_pose.cu -- the rigid-pose front end (Sec. 4.5): pairwise differences with
// the rotation-invariant length check, the rotation solve over the kept unit
// pairs, and the translation vote.
//
// Launches per problem, on the context's stream:
//   pose_count_kernel  one block per point i: the pairs (i, j > i) that pass
//            | |m| - |n| | <= mu, |m| > lmin, |n| > lmin, m = x_i - x_j,
//            n = y_i - y_j.  Decided in FP32 with an error band; a pair inside
//            the band is decided by the FP64 definition
//   pose_scan_kernel   one block: row offsets of the kept pairs
//   pose_write_kernel  one block per row: the kept pairs in lexicographic
//            order as float32 unit vectors (m/|m|, n/|n|), each from IEEE FP64
//            operations in the definition's order, so they equal the oracle's;
//            the FP64 normalisation runs on a shared-memory queue in full warps
//   (the rotation solve of the context over the kept pairs)
//   pose_tvote_kernel  t_i = y_i - R x_i in FP64 and its cell of the G^3
//            translation grid, counted in an open-addressing hash table
//   pose_tbest_kernel  one block: the cell with the largest count (ties: the
//            smallest index) and its centre
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "rv_geom.cuh"
#include "rv_runtime.h"

namespace rv {

namespace {

constexpr int kPoseThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int64_t kPoseMaxPoints = 65536;
constexpr int kPoseMaxCells = 1024;   // translation grid cells per axis
constexpr float kPoseU = 5.9604645e-8f;  // 2^-24
constexpr double kCoordMax = 1e15;    // |coordinate| limit: FP32 squares stay finite

struct PoseHdr {
    int64_t kept;                  // pairs kept
    unsigned long long rechecked;  // length checks decided in FP64
    int32_t invalid;               // a point failed validation
    int32_t pad;
    unsigned long long best_key;   // (count << 32) | (0xffffffff - cell)
    int64_t t_cell;
    int32_t t_count;
    int32_t pad2;
    double t[3];
};
static_assert(sizeof(PoseHdr) <= 256, "header slot");

struct Rot9 {
    double r[9];
};

// The definition in FP64: m = x_i - x_j, n = y_i - y_j, |m| = sqrt((m0^2 + m1^2) + m2^2).
__device__ __forceinline__ bool pose_keep64(const float *x, const float *y, int64_t i, int64_t j, double mu,
                                            double lmin, double m[3], double v[3], double *lm, double *ln) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m[c] = dsub((double)x[3 * i + c], (double)x[3 * j + c]);
        v[c] = dsub((double)y[3 * i + c], (double)y[3 * j + c]);
    }
    *lm = dsqrt(dadd(dadd(dmul(m[0], m[0]), dmul(m[1], m[1])), dmul(m[2], m[2])));
    *ln = dsqrt(dadd(dadd(dmul(v[0], v[0]), dmul(v[1], v[1])), dmul(v[2], v[2])));
    return *lm > lmin && *ln > lmin && fabs(dsub(*lm, *ln)) <= mu;
}

// The keep decision: FP32 first.  |lm32 - lm64| <= 3.1 u lm (component
// differences u, squares and sums 3u, square root), so | d32 - d64 | <= 4.1 u
// (lm + ln) for d = | |m| - |n| |; decisions within 8 u lm (lmin tests) or
// 16 u (lm + ln) (mu test) of their thresholds, plus 1e-18 for subnormal
// squares, go to FP64.
__device__ __forceinline__ bool pose_keep(const float *x, const float *y, int64_t i, int64_t j, float mu, float lmin,
                                          double mu64, double lmin64, unsigned *rechecked) {
    const float m0 = x[3 * i] - x[3 * j], m1 = x[3 * i + 1] - x[3 * j + 1], m2 = x[3 * i + 2] - x[3 * j + 2];
    const float v0 = y[3 * i] - y[3 * j], v1 = y[3 * i + 1] - y[3 * j + 1], v2 = y[3 * i + 2] - y[3 * j + 2];
    const float lm = __fsqrt_rn(fmaf(m0, m0, fmaf(m1, m1, m2 * m2)));
    const float ln = __fsqrt_rn(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
    const float d = fabsf(lm - ln);
    const float bm = 8.f * kPoseU * lm + 1e-18f, bn = 8.f * kPoseU * ln + 1e-18f;
    const float bd = 16.f * kPoseU * (lm + ln) + 1e-18f;
    if (fabsf(lm - lmin) > bm && fabsf(ln - lmin) > bn && fabsf(d - mu) > bd) return lm > lmin && ln > lmin && d <= mu;
    ++*rechecked;
    double m[3], v[3], a, b;
    return pose_keep64(x, y, i, j, mu64, lmin64, m, v, &a, &b);
}

__global__ void __launch_bounds__(kPoseThreads) pose_count_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ y, int64_t n, float mu,
                                                                  float lmin, double mu64, double lmin64,
                                                                  int32_t *__restrict__ row_count, PoseHdr *hdr) {
    const int64_t i = blockIdx.x;
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
            const float a = x[3 * i + c], b = y[3 * i + c];
            ok = ok && isfinite(a) && isfinite(b) && fabs((double)a) <= kCoordMax && fabs((double)b) <= kCoordMax;
        }
        if (!ok) atomicOr(&hdr->invalid, 1);
    }
    unsigned kept = 0, rechecked = 0;
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += kPoseThreads)
        kept += pose_keep(x, y, i, j, mu, lmin, mu64, lmin64, &rechecked);
    __shared__ unsigned wk[kPoseThreads / 32], wr[kPoseThreads / 32];
    kept = __reduce_add_sync(0xffffffffu, kept);
    rechecked = __reduce_add_sync(0xffffffffu, rechecked);
    if ((threadIdx.x & 31) == 0) {
        wk[threadIdx.x >> 5] = kept;
        wr[threadIdx.x >> 5] = rechecked;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned k = 0, r = 0;
        for (int w = 0; w < kPoseThreads / 32; ++w) {
            k += wk[w];
            r += wr[w];
        }
        row_count[i] = (int32_t)k;
        if (r) atomicAdd(&hdr->rechecked, (unsigned long long)r);
    }
}

// Exclusive prefix sums of the row counts (one block) and the total.
__global__ void __launch_bounds__(kScanThreads) pose_scan_kernel(const int32_t *__restrict__ row_count, int64_t n,
                                                                 int64_t *__restrict__ row_off, PoseHdr *hdr) {
    __shared__ int64_t part[kScanThreads];
    const int t = threadIdx.x;
    const int64_t per = (n + kScanThreads - 1) / kScanThreads;
    const int64_t b = t * per, e = min(n, b + per);
    int64_t s = 0;
    for (int64_t r = b; r < e; ++r) s += row_count[r];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {  // inclusive scan over the threads' sums
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = t ? part[t - 1] : 0;
    for (int64_t r = b; r < e; ++r) {
        row_off[r] = run;
        run += row_count[r];
    }
    if (t == kScanThreads - 1) hdr->kept = part[t];
}

// Writes row i's kept pairs at row_off[i], in increasing j.  The kept j are
// queued in shared memory and normalised in FP64 by the whole block when the
// queue fills and at the end, so FP64 work runs in full warps (a lone FP64
// lane holds its warp on GB300's narrow FP64 pipe).
constexpr int kPoseQ = 2048;

__global__ void __launch_bounds__(kPoseThreads) pose_write_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ y, int64_t n, float mu,
                                                                  float lmin, double mu64, double lmin64,
                                                                  const int64_t *__restrict__ row_off,
                                                                  float *__restrict__ a_out,
                                                                  float *__restrict__ b_out) {
    const int64_t i = blockIdx.x;
    __shared__ unsigned wcount[kPoseThreads / 32];
    __shared__ int32_t qj[kPoseQ];
    int64_t base = row_off[i];
    int qn = 0;  // queued pairs (the same in every thread)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned dummy = 0;
    auto drain = [&]() {
        for (int k = threadIdx.x; k < qn; k += kPoseThreads) {
            const int64_t j = qj[k], pos = base + k;
            double m[3], v[3], lm, ln;
            pose_keep64(x, y, i, j, mu64, lmin64, m, v, &lm, &ln);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a_out[3 * pos + c] = (float)ddiv(m[c], lm);
                b_out[3 * pos + c] = (float)ddiv(v[c], ln);
            }
        }
    };
    for (int64_t j0 = i + 1; j0 < n; j0 += kPoseThreads) {  // uniform trip count across the block
        const int64_t j = j0 + threadIdx.x;
        const bool keep = j < n && pose_keep(x, y, i, j, mu, lmin, mu64, lmin64, &dummy);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wcount[w] = __popc(bal);
        __syncthreads();
        int off = 0;
        unsigned total = 0;
        for (int k = 0; k < kPoseThreads / 32; ++k) {
            if (k < w) off += wcount[k];
            total += wcount[k];
        }
        if (keep) qj[qn + off + __popc(bal & ((1u << lane) - 1u))] = (int32_t)j;
        qn += total;
        __syncthreads();
        if (qn > kPoseQ - kPoseThreads) {
            drain();
            base += qn;
            qn = 0;
            __syncthreads();
        }
    }
    drain();
}

__device__ __forceinline__ uint32_t pose_hash(uint32_t k) {
    k ^= k >> 16;
    k *= 0x7feb352du;
    k ^= k >> 15;
    k *= 0x846ca68bu;
    k ^= k >> 16;
    return k;
}

// Translation candidates t_i = y_i - R x_i (row r: y_r - ((R_r0 x_0 + R_r1 x_1) + R_r2 x_2)) and their cells
// floor((t + L) / s) of the G^3 grid; counted per cell in an open-addressing table (key = cell + 1).
__global__ void __launch_bounds__(kPoseThreads) pose_tvote_kernel(const float *__restrict__ x,
                                                                  const float *__restrict__ y, int64_t n, Rot9 R,
                                                                  double L, double s, int G,
                                                                  uint32_t *__restrict__ tab_key,
                                                                  uint32_t *__restrict__ tab_cnt, uint32_t mask) {
    const int64_t i = (int64_t)blockIdx.x * kPoseThreads + threadIdx.x;
    if (i >= n) return;
    int64_t c3[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double rx = dadd(dadd(dmul(R.r[3 * r], (double)x[3 * i]), dmul(R.r[3 * r + 1], (double)x[3 * i + 1])),
                               dmul(R.r[3 * r + 2], (double)x[3 * i + 2]));
        const double tk = dsub((double)y[3 * i + r], rx);
        const double f = floor(ddiv(dadd(tk, L), s));
        if (!(f >= 0.0 && f < (double)G)) return;
        c3[r] = (int64_t)f;
    }
    const uint32_t key = (uint32_t)((c3[2] * G + c3[1]) * G + c3[0]) + 1u;
    uint32_t h = pose_hash(key) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {  // at most the table size: the table has room for every key
        const uint32_t k = atomicCAS(&tab_key[h], 0u, key);
        if (k == 0u || k == key) {
            atomicAdd(&tab_cnt[h], 1u);
            return;
        }
        h = (h + 1u) & mask;
    }
}

// The winning translation cell: largest count, ties to the smallest index; its centre.  One block.
__global__ void __launch_bounds__(kScanThreads) pose_tbest_kernel(const uint32_t *__restrict__ tab_key,
                                                                  const uint32_t *__restrict__ tab_cnt,
                                                                  uint32_t size, double L, double s, int G,
                                                                  PoseHdr *hdr) {
    unsigned long long best = 0;
    for (uint32_t h = threadIdx.x; h < size; h += kScanThreads) {
        const uint32_t k = tab_key[h];
        if (k) {
            const unsigned long long v = ((unsigned long long)tab_cnt[h] << 32) | (0xffffffffu - (k - 1u));
            best = v > best ? v : best;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    __shared__ unsigned long long wb[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 0; w < kScanThreads / 32; ++w) best = wb[w] > best ? wb[w] : best;
    hdr->best_key = best;
    if (best == 0) {
        hdr->t_cell = -1;
        hdr->t_count = 0;
        hdr->t[0] = hdr->t[1] = hdr->t[2] = 0.0;
        return;
    }
    const int64_t cell = (int64_t)(0xffffffffu - (uint32_t)(best & 0xffffffffull));
    const int64_t cx = cell % G, cy = (cell / G) % G, cz = cell / ((int64_t)G * G);
    hdr->t_cell = cell;
    hdr->t_count = (int32_t)(best >> 32);
    hdr->t[0] = dadd(-L, dmul(dadd((double)cx, 0.5), s));
    hdr->t[1] = dadd(-L, dmul(dadd((double)cy, 0.5), s));
    hdr->t[2] = dadd(-L, dmul(dadd((double)cz, 0.5), s));
}

bool pose_on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

void Context::pose_release() {
    if (ps_mem) {
        cudaStreamSynchronize(stream);
        cudaFree(ps_mem);
        bytes_held -= ps_cap;
    }
    ps_mem = nullptr;
    ps_cap = 0;
    if (ps_hdr_h) cudaFreeHost(ps_hdr_h);
    ps_hdr_h = nullptr;
    for (auto &e : ps_ev)
        if (e) cudaEventDestroy(e);
    ps_ev[0] = ps_ev[1] = nullptr;
}

int Context::pose_ensure(size_t need) {
    if (need <= ps_cap) return ROT_VOTE_OK;
    cudaStreamSynchronize(stream);
    if (ps_mem) {
        cudaFree(ps_mem);
        bytes_held -= ps_cap;
    }
    ps_mem = nullptr;
    ps_cap = 0;
    if (bytes_held + need > budget) return fail(ROT_VOTE_ENOMEM, "pose workspace exceeds the device memory budget");
    if (cudaMalloc(&ps_mem, need) != cudaSuccess) {
        cudaGetLastError();
        ps_mem = nullptr;
        return fail(ROT_VOTE_ENOMEM, "cudaMalloc of the pose workspace failed");
    }
    ps_cap = need;
    bytes_held += need;
    return ROT_VOTE_OK;
}

int Context::pose(const rot_vote_pose_problem *p, int np, rot_vote_pose_result *out) {
    if (!ps_hdr_h && cudaMallocHost(&ps_hdr_h, 256) != cudaSuccess) {
        cudaGetLastError();
        ps_hdr_h = nullptr;
        return fail(ROT_VOTE_ENOMEM, "pinned header allocation failed");
    }
    for (auto &ev : ps_ev)
        if (!ev && cudaEventCreate(&ev) != cudaSuccess) {
            ev = nullptr;
            return fail(ROT_VOTE_ECUDA, "creating events");
        }
    PoseHdr *hh = static_cast<PoseHdr *>(ps_hdr_h);
    for (int k = 0; k < np; ++k) {
        rot_vote_pose_result &r = out[k];
        memset(&r, 0, sizeof r);
        const rot_vote_pose_problem &P = p[k];
        const double L = P.t_half == 0.f ? 5.0 : (double)P.t_half;
        const int G = P.t_cells == 0 ? 400 : P.t_cells;
        if (!P.x || !P.y || P.n < 2 || P.n > kPoseMaxPoints || !(P.mu > 0.f) || !isfinite(P.mu) ||
            !(P.min_length >= 0.f) || !isfinite(P.min_length) || !(L > 0.0) || !isfinite(L) || G < 1 ||
            G > kPoseMaxCells || P.pairs_cap < 0 || (P.pairs_cap > 0 && (!P.pairs_a || !P.pairs_b))) {
            r.status = ROT_VOTE_EINVAL;
            last_error = "pose problem " + std::to_string(k) + ": bad argument";
            continue;
        }
        const int64_t n = P.n;
        const bool dev_in = pose_on_device(P.x) && pose_on_device(P.y);
        uint32_t tsize = 1;
        while (tsize < 2u * (uint32_t)n) tsize <<= 1;
        // layout: header | row counts | row offsets | hash keys | hash counts | staged points | kept pairs
        const size_t off_cnt = 256;
        const size_t off_off = align_up(off_cnt + sizeof(int32_t) * n, 256);
        const size_t off_tk = align_up(off_off + sizeof(int64_t) * n, 256);
        const size_t off_tc = align_up(off_tk + sizeof(uint32_t) * tsize, 256);
        const size_t off_pts = align_up(off_tc + sizeof(uint32_t) * tsize, 256);
        const size_t pts = dev_in ? 0 : align_up(sizeof(float) * 3 * n, 256);
        const size_t off_pairs = off_pts + 2 * pts;
        int rc = pose_ensure(off_pairs);
        if (rc != ROT_VOTE_OK) return rc;
        unsigned char *base = static_cast<unsigned char *>(ps_mem);
        PoseHdr *hdr = reinterpret_cast<PoseHdr *>(base);
        int32_t *row_count = reinterpret_cast<int32_t *>(base + off_cnt);
        int64_t *row_off = reinterpret_cast<int64_t *>(base + off_off);
        const float *dx = P.x, *dy = P.y;
        cudaError_t e = cudaSuccess;
        if (!dev_in) {
            float *sx = reinterpret_cast<float *>(base + off_pts), *sy = reinterpret_cast<float *>(base + off_pts + pts);
            e = cudaMemcpyAsync(sx, P.x, sizeof(float) * 3 * n, cudaMemcpyDefault, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sy, P.y, sizeof(float) * 3 * n, cudaMemcpyDefault, stream);
            dx = sx;
            dy = sy;
        }
        const float mu = P.mu, lmin = P.min_length;
        if (e == cudaSuccess) e = cudaEventRecord(ps_ev[0], stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(PoseHdr), stream);
        if (e == cudaSuccess) {
            pose_count_kernel<<<(unsigned)n, kPoseThreads, 0, stream>>>(dx, dy, n, mu, lmin, (double)mu, (double)lmin,
                                                                         row_count, hdr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            pose_scan_kernel<<<1, kScanThreads, 0, stream>>>(row_count, n, row_off, hdr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hh, hdr, sizeof(PoseHdr), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "running the pose pair count");
        r.pairs_tested = n * (n - 1) / 2;
        r.pairs_kept = hh->kept;
        r.pairs_rechecked = (int64_t)hh->rechecked;
        if (hh->invalid) {
            r.status = ROT_VOTE_EINVAL;
            last_error = "pose problem " + std::to_string(k) + ": non-finite or out-of-range coordinate";
            continue;
        }
        const int64_t K = hh->kept;
        // the kept pairs: grow the workspace (the count pass fixed K), then write them
        const size_t need = off_pairs + 2 * align_up(sizeof(float) * 3 * (size_t)std::max<int64_t>(K, 1), 256);
        if (need > ps_cap) {
            if (!dev_in) {  // the staged points move with the workspace: stage them again after growing
                rc = pose_ensure(need);
                if (rc != ROT_VOTE_OK) return rc;
                base = static_cast<unsigned char *>(ps_mem);
                float *sx = reinterpret_cast<float *>(base + off_pts), *sy = reinterpret_cast<float *>(base + off_pts + pts);
                e = cudaMemcpyAsync(sx, P.x, sizeof(float) * 3 * n, cudaMemcpyDefault, stream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(sy, P.y, sizeof(float) * 3 * n, cudaMemcpyDefault, stream);
                dx = sx;
                dy = sy;
            } else {
                rc = pose_ensure(need);
                if (rc != ROT_VOTE_OK) return rc;
                base = static_cast<unsigned char *>(ps_mem);
            }
            // the row offsets died with the old workspace: recount
            hdr = reinterpret_cast<PoseHdr *>(base);
            row_count = reinterpret_cast<int32_t *>(base + off_cnt);
            row_off = reinterpret_cast<int64_t *>(base + off_off);
            if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(PoseHdr), stream);
            if (e == cudaSuccess) {
                pose_count_kernel<<<(unsigned)n, kPoseThreads, 0, stream>>>(dx, dy, n, mu, lmin, (double)mu,
                                                                             (double)lmin, row_count, hdr);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                pose_scan_kernel<<<1, kScanThreads, 0, stream>>>(row_count, n, row_off, hdr);
                e = cudaGetLastError();
            }
        }
        float *pa = reinterpret_cast<float *>(base + off_pairs);
        float *pb = reinterpret_cast<float *>(base + off_pairs + align_up(sizeof(float) * 3 * (size_t)std::max<int64_t>(K, 1), 256));
        if (e == cudaSuccess && K > 0) {
            pose_write_kernel<<<(unsigned)n, kPoseThreads, 0, stream>>>(dx, dy, n, mu, lmin, (double)mu, (double)lmin,
                                                                         row_off, pa, pb);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ps_ev[1], stream);
        if (e == cudaSuccess && P.pairs_cap > 0 && K > 0) {
            const size_t m = (size_t)std::min<int64_t>(K, P.pairs_cap);
            e = cudaMemcpyAsync(P.pairs_a, pa, sizeof(float) * 3 * m, cudaMemcpyDefault, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(P.pairs_b, pb, sizeof(float) * 3 * m, cudaMemcpyDefault, stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "writing the pose pairs");
        float ms_front = 0.f;
        cudaEventElapsedTime(&ms_front, ps_ev[0], ps_ev[1]);
        // the rotation: the context's solve over the kept unit pairs
        if (K >= 2) {
            rot_vote_problem rp;
            memset(&rp, 0, sizeof rp);
            rp.a = pa;
            rp.b = pb;
            rp.n = K;
            rp.delta = P.delta;
            rp.grid_n = P.grid_n;
            rp.levels = P.levels;
            rc = solve(&rp, 1, &r.rot);
            if (rc != ROT_VOTE_OK) return rc;
        } else {
            r.rot.status = ROT_VOTE_EDEGENERATE;
        }
        if (r.rot.status != ROT_VOTE_OK && r.rot.status != ROT_VOTE_EDEGENERATE) {
            r.status = r.rot.status;
            continue;
        }
        if (K < 2) {
            r.status = ROT_VOTE_EDEGENERATE;
            r.t_cell = -1;
            continue;
        }
        // the translation vote with the solved rotation
        Rot9 R;
        for (int c = 0; c < 9; ++c) R.r[c] = r.rot.R[c];
        const double s = (2.0 * L) / (double)G;
        uint32_t *tk = reinterpret_cast<uint32_t *>(base + off_tk), *tc = reinterpret_cast<uint32_t *>(base + off_tc);
        e = cudaEventRecord(ps_ev[0], stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(tk, 0, sizeof(uint32_t) * tsize, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(tc, 0, sizeof(uint32_t) * tsize, stream);
        if (e == cudaSuccess) {
            pose_tvote_kernel<<<(unsigned)((n + kPoseThreads - 1) / kPoseThreads), kPoseThreads, 0, stream>>>(
                dx, dy, n, R, L, s, G, tk, tc, tsize - 1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            pose_tbest_kernel<<<1, kScanThreads, 0, stream>>>(tk, tc, tsize, L, s, G, hdr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ps_ev[1], stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hh, hdr, sizeof(PoseHdr), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "running the translation vote");
        float ms_t = 0.f;
        cudaEventElapsedTime(&ms_t, ps_ev[0], ps_ev[1]);
        for (int c = 0; c < 3; ++c) r.t[c] = hh->t[c];
        r.t_cell = hh->t_cell;
        r.t_count = hh->t_count;
        r.status = r.rot.status;
        r.ms_gpu = ms_front + ms_t;
    }
    return ROT_VOTE_OK;
}

}  // namespace rv

extern "C" int rot_vote_pose(rot_vote_ctx *ctx, const rot_vote_pose_problem *p, int n_problems,
                             rot_vote_pose_result *out) {
    if (!ctx || !p || !out || n_problems < 1) return ROT_VOTE_EINVAL;
    rv::Context *c = reinterpret_cast<rv::Context *>(ctx);
    std::lock_guard<std::mutex> g(c->launch_mu);
    return c->pose(p, n_problems, out);
}
