// rv_static.cu -- rot_vote_count_cells_static: the FP32 vote of a caller-given
// cell list with every scratch buffer in one file-scope static device array,
// so the call allocates no device memory.
//
// The call runs five launches on the caller's stream: a set-up kernel (header,
// work lists, cell table, counts zeroed), the pair step (launch_pair_prep), the
// CUDA-core FP32 vote (launch_vote_simt) and its FP64 resolution pass
// (launch_resolve64: two kernels), the kernels a solve runs, here with their pair pool, cell
// table, work lists and FP64 queue in the static array.  It then reads back two
// flags (invalid pairs, invalid cells) and returns.
#include <mutex>

#include "rv_geom.cuh"
#include "rv_internal.h"

namespace rv {

namespace {

constexpr int64_t kStaticMaxPairs = ROT_VOTE_STATIC_MAX_PAIRS;
constexpr int64_t kStaticMaxCells = ROT_VOTE_STATIC_MAX_CELLS;
constexpr int kStaticPairChunk = 2048;  // pairs per vote work item (multiple of kPairTile)
constexpr int64_t kStaticMaxTiles = kStaticMaxPairs / kPairTile;
constexpr int64_t kStaticMaxItems =
    ((kStaticMaxCells + kSimtItemCells - 1) / kSimtItemCells) * (kStaticMaxPairs / kStaticPairChunk);
static_assert(kStaticMaxPairs % kStaticPairChunk == 0 && kStaticPairChunk % kPairTile == 0, "pair limits");

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the buffers inside the scratch array (each 256-aligned).
constexpr size_t kOffProb = 0;
constexpr size_t kOffLevel = 256;
constexpr size_t kOffStats = 512;
constexpr size_t kOffFlags = 768;  // int32 ncells, bad_cell, FP64-queue length, queue-full flag
constexpr size_t kOffTiles = 1024;
constexpr size_t kOffItems = al256(kOffTiles + sizeof(int2) * kStaticMaxTiles);
constexpr size_t kOffS32 = al256(kOffItems + sizeof(VoteItem) * kStaticMaxItems);
constexpr size_t kOffPr = al256(kOffS32 + sizeof(float4) * 3 * kStaticMaxPairs);
constexpr size_t kOffQ = al256(kOffPr + sizeof(float4) * 2 * kStaticMaxPairs);
constexpr size_t kOffChord = al256(kOffQ + sizeof(double4_32a) * kStaticMaxCells);
constexpr size_t kOffTrig = al256(kOffChord + sizeof(double) * kStaticMaxCells);
constexpr size_t kOffIdx = al256(kOffTrig + sizeof(double2) * kStaticMaxCells);
constexpr size_t kOffM32 = al256(kOffIdx + sizeof(int64_t) * kStaticMaxCells);
constexpr size_t kOffR32 = al256(kOffM32 + sizeof(float4) * 3 * kStaticMaxCells);
constexpr int kStaticAmbCap = 8192;  // tests within 2e-6 of the threshold (about 1100 expected at the limits)
constexpr size_t kOffAmb = al256(kOffR32 + sizeof(float4) * 3 * kStaticMaxCells);
constexpr size_t kOffEnd = al256(kOffAmb + sizeof(Amb64) * kStaticAmbCap);
static_assert(sizeof(ProbRef) <= 256 && sizeof(LevelRef) <= 256 && sizeof(ProbStats) <= 256, "header slots");
static_assert(kOffEnd <= (size_t)ROT_VOTE_STATIC_SCRATCH_BYTES, "static scratch layout exceeds its size");

// The scratch.  In host code this name is only a handle for
// cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_static_scratch[ROT_VOTE_STATIC_SCRATCH_BYTES];

struct StaticArgs {
    unsigned char *base;  // device address of g_static_scratch
    const float *a, *b;
    const int64_t *cells;
    int32_t *counts;
    int64_t n, npad;
    int32_t ncells, grid_n;
    int32_t ntiles, nitems, cell_items, pair_chunks;
    double sin_d, cos_d;
    float delta;
};

__device__ __forceinline__ CellSoA static_cells(unsigned char *base) {
    CellSoA c;
    c.q = reinterpret_cast<double4_32a *>(base + kOffQ);
    c.chord = reinterpret_cast<double *>(base + kOffChord);
    c.trig = reinterpret_cast<double2 *>(base + kOffTrig);
    c.idx = reinterpret_cast<int64_t *>(base + kOffIdx);
    c.m32 = reinterpret_cast<float4 *>(base + kOffM32);
    c.R32 = reinterpret_cast<float4 *>(base + kOffR32);
    return c;
}

// Writes the header, the work lists and the cell table, and zeroes the
// counts.  Everything a previous call left in the array is overwritten
// before it is read, except the bad-cell flag, which the host clears first.
__global__ void static_setup_kernel(StaticArgs A) {
    unsigned char *base = A.base;
    const CellSoA cells = static_cells(base);
    int32_t *flags = reinterpret_cast<int32_t *>(base + kOffFlags);
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            ProbRef P;
            P.a = A.a;
            P.b = A.b;
            P.n = A.n;
            P.pool_off = 0;
            P.sin_d = A.sin_d;
            P.cos_d = A.cos_d;
            P.delta = A.delta;
            P.levels = 0;
            P.grid_n = A.grid_n;
            *reinterpret_cast<ProbRef *>(base + kOffProb) = P;
            LevelRef L;
            L.cells = cells;
            L.ncells = flags;
            L.counts = A.counts;
            L.cap = A.ncells;
            L.n_side = A.grid_n;
            L.chart = 0;
            *reinterpret_cast<LevelRef *>(base + kOffLevel) = L;
            ProbStats S;
            S.tests = 0;
            S.rechecked = 0;
            S.ambiguous = 0;
            S.resolved = 0;
            S.invalid = 0;
            S.pad = 0;
            *reinterpret_cast<ProbStats *>(base + kOffStats) = S;
            flags[0] = A.ncells;
        }
        int2 *tiles = reinterpret_cast<int2 *>(base + kOffTiles);
        for (int t = threadIdx.x; t < A.ntiles; t += blockDim.x) tiles[t] = make_int2(0, t);
        VoteItem *items = reinterpret_cast<VoteItem *>(base + kOffItems);
        for (int k = threadIdx.x; k < A.nitems; k += blockDim.x) {
            const int ci = k / A.pair_chunks, pc = k % A.pair_chunks;
            VoteItem W;
            W.prob = 0;
            W.cell_begin = ci * kSimtItemCells;
            W.pair_begin = pc * kStaticPairChunk;
            W.pair_end = (int32_t)min((int64_t)(pc + 1) * kStaticPairChunk, A.npad);
            items[k] = W;
        }
    }
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= A.ncells) return;
    const int64_t n = A.grid_n, idx = A.cells[pos];
    const int64_t ix = idx % n, iy = (idx / n) % n, iz = idx / (n * n);
    if (idx >= 0 && idx < n * n * n && cell_exists(A.grid_n, ix, iy, iz)) {
        write_cell(cells, pos, A.grid_n, 0, ix, iy, iz);
    } else {  // reported as EINVAL (counts then unspecified); the slot gets a placeholder record
        atomicOr(&flags[1], 1);
        cells.q[pos] = make_double4_32a(1.0, 0.0, 0.0, 0.0);
        cells.chord[pos] = 0.0;
        cells.trig[pos] = make_double2(1.0, 0.0);
        cells.idx[pos] = idx;
        for (int k = 0; k < 3; ++k) cells.m32[3 * pos + k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < 3; ++k) cells.R32[3 * pos + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    A.counts[pos] = 0;
}

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
unsigned char *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t static_base(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

// Memory the kernels on device `dev` may read and write: that device's own
// memory, or managed memory.
bool device_accessible(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

}  // namespace rv

extern "C" int rot_vote_count_cells_static(const float *a, const float *b, int64_t n, double delta, int grid_n,
                                           const int64_t *cells, int32_t ncells, int32_t *counts,
                                           void *cuda_stream) {
    using namespace rv;
    if (!a || !b || !cells || !counts) return ROT_VOTE_EINVAL;
    if (n < 2 || ncells < 1) return ROT_VOTE_EINVAL;
    if (n > kStaticMaxPairs || ncells > kStaticMaxCells) return ROT_VOTE_ETOOLARGE;
    if (!(delta > 0.0) || !(delta < 1.5707963)) return ROT_VOTE_EINVAL;
    if (grid_n < 2 || grid_n > (1 << 20) || (grid_n & (grid_n - 1)) != 0) return ROT_VOTE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ROT_VOTE_ECUDA;
    if (!device_accessible(a, dev) || !device_accessible(b, dev) || !device_accessible(cells, dev) ||
        !device_accessible(counts, dev))
        return ROT_VOTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    if (static_base(&base) != cudaSuccess) return ROT_VOTE_ECUDA;

    StaticArgs A;
    A.base = base;
    A.a = a;
    A.b = b;
    A.cells = cells;
    A.counts = counts;
    A.n = n;
    A.npad = (n + kPairTile - 1) / kPairTile * kPairTile;
    A.ncells = ncells;
    A.grid_n = grid_n;
    A.ntiles = (int32_t)(A.npad / kPairTile);
    A.cell_items = (ncells + kSimtItemCells - 1) / kSimtItemCells;
    A.pair_chunks = (int32_t)((A.npad + kStaticPairChunk - 1) / kStaticPairChunk);
    A.nitems = A.cell_items * A.pair_chunks;
    const float df = (float)delta;  // the pair step and the tables take delta as float, as a solve does
    A.delta = df;
    A.sin_d = sin((double)df);
    A.cos_d = cos((double)df);

    cudaError_t e = cudaMemsetAsync(base + kOffFlags + sizeof(int32_t), 0, 3 * sizeof(int32_t), s);
    const int threads = 256;
    const int blocks = (ncells + threads - 1) / threads;
    if (e == cudaSuccess) {
        static_setup_kernel<<<blocks, threads, 0, s>>>(A);
        e = cudaGetLastError();
    }
    ProbRef *probs = reinterpret_cast<ProbRef *>(base + kOffProb);
    LevelRef *lref = reinterpret_cast<LevelRef *>(base + kOffLevel);
    ProbStats *stats = reinterpret_cast<ProbStats *>(base + kOffStats);
    PairPool pool;
    pool.p32 = reinterpret_cast<float4 *>(base + kOffS32);
    pool.pr = reinterpret_cast<float4 *>(base + kOffPr);
    pool.tcb = nullptr;
    pool.tc_k = 0;
    if (e == cudaSuccess)
        e = launch_pair_prep(probs, reinterpret_cast<const int2 *>(base + kOffTiles), A.ntiles, pool, ROT_PREC_FP32,
                             stats, s);
    AmbQueue amb;
    amb.q = reinterpret_cast<Amb64 *>(base + kOffAmb);
    amb.count = reinterpret_cast<int *>(base + kOffFlags) + 2;
    amb.ovf = reinterpret_cast<int *>(base + kOffFlags) + 3;
    amb.cap = kStaticAmbCap;
    if (e == cudaSuccess)
        e = launch_vote_simt(reinterpret_cast<const VoteItem *>(base + kOffItems), A.nitems, probs, lref, 1, 0, pool,
                             stats, 4, A.nitems, nullptr, amb, s);
    if (e == cudaSuccess) e = launch_resolve64(amb, probs, 1, lref, 1, 0, pool, stats, 2 * kStaticMaxCells / 256, s);
    // header slots back to the host: ProbStats.invalid and the bad-cell flag
    unsigned char hdr[1024];
    if (e == cudaSuccess) e = cudaMemcpyAsync(hdr, base, sizeof hdr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ROT_VOTE_ECUDA;
    const ProbStats *hs = reinterpret_cast<const ProbStats *>(hdr + kOffStats);
    const int32_t *hf = reinterpret_cast<const int32_t *>(hdr + kOffFlags);
    if (hs->invalid || hf[1]) return ROT_VOTE_EINVAL;
    return ROT_VOTE_OK;
}
