// ORAS sweeps on the fifth-generation tensor cores (tcgen05, sm_103a): the
// multifrontal forward and backward products of sweep.cu (the B_i^{-1} of
// Eq. ORAS applied to m right-hand sides at once, Section 3), with the factor
// panels streamed by bulk asynchronous copies into shared memory and the
// products accumulated in tensor memory.
//
// Factor layout ("tiled panels", written once per factorisation by
// pack_tiled_kernel).  The TF32 form of tcgen05.mma reads both operands
// K-major (K contiguous in a line), and the two sweeps contract a front's
// f x p partitioned-inverse panel [L11^{-1}; -L21 L11^{-1}] over different
// indices -- the forward product over pivots, the backward one over rows --
// so the panel is stored twice, cut into 8 x 8 blocks (rows and pivots padded
// to multiples of 8 with zeros).  A block is two 256-byte planes (real parts,
// then imaginary parts), each 8 lines of 32 bytes in the 32-byte swizzled
// order of the tensor cores (16-byte chunk j of line r at chunk
// j ^ ((r >> 2) & 1)):
//   - forward copy: line = front row, 8 floats = pivots; blocks ordered
//     [pivot chunk][row group][plane], so one 8-pivot K step of a 128-row
//     tile is 16 consecutive blocks (row groups at the stride-byte offset);
//   - backward copy: line = pivot, 8 floats = front rows; blocks ordered
//     [row chunk][pivot group][plane].
// A stage of 32 K values is at most four contiguous byte ranges, copied with
// cp.async.bulk.  The right-hand sides are written K-major into the B stage by
// the gather warps (line = real column, 32 floats = the stage's K rows,
// 128-byte swizzle).
//
// Complex product as two real products.  With A = Ar + i Ai (the two planes)
// and the right-hand sides B stored as reals [k][2c + (0 re, 1 im)], the MMA
// computes Dr = Ar B and Di = Ai B (N = 64 real columns for 32 complex
// columns, TF32 inputs -- the tensor core reads the FP32 bits and drops the
// low 13 mantissa bits -- FP32 accumulation); then
//   Re C(i, c) = Dr[i][2c] - Di[i][2c+1],  Im C(i, c) = Dr[i][2c+1] + Di[i][2c].
//
// Kernel: persistent, two CTAs per SM, tiles (front, 128-row tile, 32-column
// chunk) taken in a fixed stride.  Warp roles:
//   warp 0      bulk copies: lanes 0-3 the panel blocks, the right-hand-side
//               rows into the stage's staging rows (one copy per run of
//               rows that are contiguous in memory, else one per row; the
//               update-row indices of the backward product looked up by
//               the lanes first), one mbarrier transaction count
//   warp 1      owns the tensor memory (2 x 128 columns: accumulators double
//               buffered across tiles); one lane issues tcgen05.mma and commits
//   warps 2-3   transpose the staging rows into the K-major B tile (shared
//               memory only)
//   warps 4-7   epilogue: tcgen05.ld, complex combine, D^{-1} scaling or
//               extend-add of the children's update rows, global stores
// Stages (2 x 48 KB per CTA, two CTAs per SM) form a ring shared by all tiles
// of the CTA, so loads of the next tile overlap the products and the epilogue
// of the current one; no
// thread waits on device memory inside a stage except the copy lanes' index
// lookups.  The right-hand-side rows move by 16-byte-aligned bulk copies, so
// the engine needs an even number of columns (the solver falls back to the
// mma.sync engine otherwise).
// Every wait is bounded: on expiry the kernel records an error code, the
// other roles stop at their next wait, and the CTA frees its tensor memory
// and returns.
#include <algorithm>

#include "common.h"
#include "kernels.h"

namespace mwi {
namespace {

constexpr int kStages = 2;                  // stage ring per CTA (two CTAs per SM)
constexpr int kCtasPerSm = 2;
constexpr int kUrCache = 1024;              // update-row indices of a backward tile kept in shared memory
constexpr int kKS = 4;                      // K chunks of 8 per stage (K = 32)
constexpr int kAStage = 32768;              // 4 K chunks x 16 groups of 8 M lines x 2 planes x 256 B
constexpr int kBStage = 8192;               // 64 real columns x 32 K floats
constexpr int kStage = kAStage + 2 * kBStage;  // + the staging rows [32][nc complex] of the copies
constexpr int kThreads = 256;
constexpr int kTmemCols = 256;
constexpr int kSmemBytes = kStages * kStage + 1024 /* barriers */ + kUrCache * 4 + 1024 /* alignment */;
static_assert(kSmemBytes * kCtasPerSm <= 228 * 1024 - 2048, "shared memory per SM");
constexpr long long kWaitLimit = 1ll << 24;

enum { kFwdT = 0, kBwdT = 1 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on a phase; false if the CTA aborts or the limit expires
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        if (mbar_try(bar, parity)) return true;  // try_wait suspends in hardware for a while
        if (*abort_flag) return false;
        if (it > (1 << 20)) __nanosleep(256);
    }
    *abort_flag = 1;
    atomicExch(err, code);
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor of a K-major operand: start, leading /
// stride byte offsets (>> 4; the leading offset is unused by swizzled K-major
// layouts), version 1 (bit 46), layout type at bits 61-63 (2 = 128-byte
// swizzle, 6 = 32-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)layout << 61;
    return d;
}
constexpr uint32_t kSw128 = 2, kSw32 = 6;

// instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Tile geometry shared by every role.  Forward: M = front rows row0..
// (row groups g0.., ng of them), K = pivots [0, min(p, row0 + 128)) in chunks
// of 8.  Backward: M = pivots row0.. (pivot groups g0..), K = front rows from
// row0 (the panel is zero above its diagonal) to f, in chunks of 8.  The
// chunks of a front's copy are cstride blocks apart.
struct TcGeom {
    int p, f, row0, g0, ng, k0, nk, nst, cstride;
};

template <int MODE>
__device__ __forceinline__ TcGeom tc_geom(const TileDesc& d) {
    TcGeom g;
    g.p = d.p;
    g.f = d.f;
    g.row0 = d.row0;
    const int F8 = (d.f + 7) >> 3, P8 = (d.p + 7) >> 3;
    g.g0 = d.row0 >> 3;
    if (MODE == kFwdT) {
        g.ng = min(16, F8 - g.g0);
        g.k0 = 0;
        g.nk = (min(d.p, d.row0 + 128) + 7) >> 3;
        g.cstride = F8;
    } else {
        g.ng = min(16, P8 - g.g0);
        g.k0 = d.row0 >> 3;
        g.nk = F8 - g.k0;
        g.cstride = P8;
    }
    g.nst = (g.nk + kKS - 1) / kKS;
    return g;
}

// number of the stage's 32 K rows that hold data (the rest of the B tile is zero)
template <int MODE>
__device__ __forceinline__ int stage_rows(const TcGeom& G, int st) {
    const int lim = MODE == kFwdT ? min(G.p, G.row0 + 128) - st * 32 : G.f - (G.row0 + st * 32);
    return max(0, min(32, lim));
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) sweep_tc_kernel(
    const TileDesc* __restrict__ tiles, int ntiles, int nchunks, const int32_t* __restrict__ urows,
    const int2* __restrict__ asm2, const float* __restrict__ wt, const float2* __restrict__ dinv,
    float2* __restrict__ Y, float2* __restrict__ Z, float2* __restrict__ upd, int m, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
    // bars: raw[kStages] (copies landed), full[kStages] (B tile ready), empty[kStages]
    // (stage consumed), tfull[2], tempty[2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kStages + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int32_t* sur = reinterpret_cast<int32_t*>(smem + kStages * kStage + 1024);  // copy warp's index cache
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    auto raw_bar = [&](int s) { return smem_u32(bars + s); };
    auto full_bar = [&](int s) { return smem_u32(bars + kStages + s); };
    auto empty_bar = [&](int s) { return smem_u32(bars + 2 * kStages + s); };
    auto tfull_bar = [&](int b) { return smem_u32(bars + 3 * kStages + b); };
    auto tempty_bar = [&](int b) { return smem_u32(bars + 3 * kStages + 2 + b); };

    // stale shared memory must be finite: the MMA reads whole blocks, and the
    // zero right-hand-side rows only cancel finite factor entries
    for (int i = threadIdx.x; i < kStages * kStage / 16; i += kThreads)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    fence_proxy_async();
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(raw_bar(s), 1);       // the copy lane, with the stage's transaction bytes
            mbar_init(full_bar(s), 2);      // the 2 transpose warps
            mbar_init(empty_bar(s), 1);     // tcgen05.commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), 4);    // the 4 epilogue warps
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int total = ntiles * nchunks;

    if (warp == 0) {
        // ---------------- bulk copies: panel blocks (lane 0) and one
        // right-hand-side row per lane into the stage's staging rows
        long long g = 0;
        bool ok = true;
        for (int ti = blockIdx.x; ti < total && ok; ti += gridDim.x) {
            const TileDesc d = tiles[ti / nchunks];
            const TcGeom G = tc_geom<MODE>(d);
            const int c0 = (ti % nchunks) * 32, nc = min(32, m - c0);
            const uint32_t row_bytes = (uint32_t)nc * 8u;
            const float* P = wt + d.a_off;
            const int32_t* ur = urows + d.u_off;
            // backward: the tile's update-row indices (at most kUrCache) into shared
            // memory, one coalesced pass; the stages then look them up there
            const int u = G.f - G.p;
            const bool ur_cached = MODE == kBwdT && u <= kUrCache;
            __syncwarp();
            if (ur_cached) {
                // eight loads in flight per lane before their stores
                for (int j0 = 0; j0 < u; j0 += 256) {
                    int v[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int j = j0 + 32 * t + lane;
                        v[t] = j < u ? ur[j] : 0;
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int j = j0 + 32 * t + lane;
                        if (j < u) sur[j] = v[t];
                    }
                }
                __syncwarp();
            }
            for (int st = 0; st < G.nst; ++st, ++g) {
                const int s = (int)(g % kStages);
                const uint32_t ph = (uint32_t)((g / kStages) & 1);
                // the source row of this lane, looked up before the stage is free
                const int nv = stage_rows<MODE>(G, st);
                const float2* src = nullptr;
                if (lane < nv) {
                    if (MODE == kFwdT) {
                        src = Y + (d.rowbase + st * 32 + lane) * m + c0;
                    } else {
                        const int i = G.row0 + st * 32 + lane;
                        src = i < G.p ? Z + (d.rowbase + i) * m + c0
                                      : Y + (d.sbase + (ur_cached ? sur[i - G.p] : ur[i - G.p])) * m + c0;
                    }
                }
                if (lane == 0) ok = mbar_wait(empty_bar(s), ph ^ 1, abort_flag, err, 1);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                const uint32_t a_dst = sbase + s * kStage;
                const int k0 = G.k0 + st * kKS, nk = min(kKS, G.k0 + G.nk - k0);
                const uint32_t a_bytes = (uint32_t)G.ng * 512u;
                if (lane == 0) mbar_arrive_tx(raw_bar(s), a_bytes * nk + row_bytes * nv);
                __syncwarp();
                if (lane < nk)
                    bulk_g2s(a_dst + lane * 8192, P + ((int64_t)(k0 + lane) * G.cstride + G.g0) * 128, a_bytes,
                             raw_bar(s));
                // right-hand-side rows: with one column chunk (nc = m) consecutive rows are
                // contiguous in memory, so each run of consecutive source rows moves as one
                // copy (the forward pivot rows are one run; the backward rows a few)
                const unsigned long long sa = reinterpret_cast<unsigned long long>(src);
                const unsigned long long prev = __shfl_up_sync(0xffffffffu, sa, 1);
                const bool lead = lane < nv && (nchunks > 1 || lane == 0 || sa != prev + row_bytes);
                const unsigned leaders = __ballot_sync(0xffffffffu, lead);
                if (lead) {
                    const unsigned later = leaders & ~((2u << lane) - 1u);
                    const int len = (later ? __ffs(later) - 1 : nv) - lane;
                    bulk_g2s(a_dst + kAStage + kBStage + lane * row_bytes, src, row_bytes * (uint32_t)len, raw_bar(s));
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- tensor-core products
        if (lane == 0) {
            long long g = 0;
            int it = 0;
            bool ok = true;
            constexpr uint32_t kIdesc = idesc_tf32(128, 64);
            for (int ti = blockIdx.x; ti < total && ok; ti += gridDim.x, ++it) {
                const TileDesc d = tiles[ti / nchunks];
                const TcGeom G = tc_geom<MODE>(d);
                const int buf = it & 1;
                if (!(ok = mbar_wait(tempty_bar(buf), ((it >> 1) & 1) ^ 1, abort_flag, err, 2))) break;
                tc_fence_after();
                const uint32_t dr = tmem + buf * 128, di = dr + 64;
                for (int st = 0; st < G.nst; ++st, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t ph = (uint32_t)((g / kStages) & 1);
                    if (!(ok = mbar_wait(full_bar(s), ph, abort_flag, err, 3))) break;
                    tc_fence_after();
                    const uint32_t a0 = sbase + s * kStage, b0 = a0 + kAStage;
                    const int nk = min(kKS, G.nk - st * kKS);
                    for (int c = 0; c < nk; ++c) {
                        // B: 64 lines (real columns) of 128 B, K step c = bytes 32c of every line
                        const uint64_t bd = smem_desc(b0 + c * 32, 1024, kSw128);
                        const uint32_t acc = (st > 0 || c > 0) ? 1u : 0u;
                        mma_tf32(dr, smem_desc(a0 + c * 8192, 512, kSw32), bd, kIdesc, acc);
                        mma_tf32(di, smem_desc(a0 + c * 8192 + 256, 512, kSw32), bd, kIdesc, acc);
                    }
                    mma_commit(empty_bar(s));
                }
                if (!ok) break;
                mma_commit(tfull_bar(buf));
            }
        }
    } else if (warp < 4) {
        // ---------------- staging rows [32][nc complex] -> K-major B tile
        // (line = real column, 32 K floats, 128-byte swizzle); thread: column
        // `lane`, four groups of 4 rows
        const int rg = warp - 2;
        long long g = 0;
        bool ok = true;
        for (int ti = blockIdx.x; ti < total && ok; ti += gridDim.x) {
            const TileDesc d = tiles[ti / nchunks];
            const TcGeom G = tc_geom<MODE>(d);
            const int nc = min(32, m - (ti % nchunks) * 32);  // columns of the chunk (staging row length)
            const bool cin = lane < nc;
            for (int st = 0; st < G.nst; ++st, ++g) {
                const int s = (int)(g % kStages);
                const uint32_t ph = (uint32_t)((g / kStages) & 1);
                if (!(ok = mbar_wait(raw_bar(s), ph, abort_flag, err, 4))) break;
                const int nv = stage_rows<MODE>(G, st);
                unsigned char* B = smem + s * kStage + kAStage;
                const float2* R = reinterpret_cast<const float2*>(B + kBStage);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int q = rg * 4 + h;  // rows 4q .. 4q+3
                    float2 v[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int r = 4 * q + j;
                        v[j] = (cin && r < nv) ? R[r * nc + lane] : make_float2(0.f, 0.f);
                    }
                    const int n0 = 2 * lane;
                    *reinterpret_cast<float4*>(B + (n0 >> 3) * 1024 + (n0 & 7) * 128 + ((q ^ (n0 & 7)) << 4)) =
                        make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
                    const int n1 = n0 + 1;
                    *reinterpret_cast<float4*>(B + (n1 >> 3) * 1024 + (n1 & 7) * 128 + ((q ^ (n1 & 7)) << 4)) =
                        make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full_bar(s));
            }
        }
    } else {
        // ---------------- epilogue
        const int lg = warp & 3;  // tensor-memory lane group of this warp
        const int i = lg * 32 + lane;
        int it = 0;
        bool ok = true;
        for (int ti = blockIdx.x; ti < total && ok; ti += gridDim.x, ++it) {
            const TileDesc d = tiles[ti / nchunks];
            const int c0 = (ti % nchunks) * 32;
            const int buf = it & 1;
            // loads that do not depend on the product, issued before waiting for it
            const int gi = d.row0 + i;
            float2 dv = make_float2(0.f, 0.f);
            int2 src = make_int2(-1, -1);
            if (MODE == kFwdT) {
                if (gi < d.p) dv = dinv[d.rowbase + gi];
                else if (gi < d.f) src = asm2[d.asm_base + gi];
            }
            if (!(ok = mbar_wait(tfull_bar(buf), (it >> 1) & 1, abort_flag, err, 5))) break;
            tc_fence_after();
            const uint32_t t0 = tmem + ((uint32_t)(lg * 32) << 16) + buf * 128;
            const int nc = min(32, m - c0);
            float2* dst = nullptr;
            if (MODE == kBwdT) {
                if (gi < d.p) dst = Y + (d.rowbase + gi) * m + c0;
            } else if (gi < d.p) {
                dst = Z + (d.rowbase + gi) * m + c0;
            } else if (gi < d.f) {
                dst = upd + (d.upd_row + gi - d.p) * m + c0;
            }
            const bool vec = nc == 32 && (m & 1) == 0;
            // two halves of 16 complex columns: tensor-memory loads, combine,
            // D^{-1} or the children's rows, stores; the accumulator is released
            // once the second half is in registers
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float o[32];
                {
                    float dr[32], di[32];
                    tmem_ld32(t0 + h * 32, dr);
                    tmem_ld32(t0 + 64 + h * 32, di);
                    tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        o[2 * q] = dr[2 * q] - di[2 * q + 1];
                        o[2 * q + 1] = dr[2 * q + 1] + di[2 * q];
                    }
                }
                if (h == 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty_bar(buf));
                }
                if (!dst) continue;
                const int cb = 16 * h;  // first complex column of the half
                if (MODE == kFwdT && gi < d.p) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float re = o[2 * q], im = o[2 * q + 1];
                        o[2 * q] = re * dv.x - im * dv.y;
                        o[2 * q + 1] = re * dv.y + im * dv.x;
                    }
                } else if (MODE == kFwdT) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int sr = k ? src.y : src.x;
                        if (sr < 0) continue;
                        const float2* a = upd + (int64_t)sr * m + c0 + cb;
                        if (vec) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 v = reinterpret_cast<const float4*>(a)[q];
                                o[4 * q] += v.x;
                                o[4 * q + 1] += v.y;
                                o[4 * q + 2] += v.z;
                                o[4 * q + 3] += v.w;
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                if (cb + q < nc) {
                                    const float2 v = a[q];
                                    o[2 * q] += v.x;
                                    o[2 * q + 1] += v.y;
                                }
                        }
                    }
                }
                if (vec) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        reinterpret_cast<float4*>(dst + cb)[q] =
                            make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (cb + q < nc) dst[cb + q] = make_float2(o[2 * q], o[2 * q + 1]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// One block per (front, 32-row block): the block's panel rows, for every
// 8-pivot chunk, into both tiled copies (layout in the header comment).
__device__ __forceinline__ int swz32(int line, int e) { return line * 8 + ((((e >> 2) ^ ((line >> 2) & 1)) << 2) | (e & 3)); }

__global__ void __launch_bounds__(256) pack_tiled_kernel(const int2* __restrict__ blocks,
                                                         const int64_t* __restrict__ f_off,
                                                         const int64_t* __restrict__ t_off,
                                                         const int32_t* __restrict__ P, const int32_t* __restrict__ U,
                                                         const float2* __restrict__ ws, float* __restrict__ wt,
                                                         int64_t bwd_base) {
    const int2 bl = blocks[blockIdx.x];  // (front, 32-row block)
    const int s = bl.x;
    const int p = P[s], f = p + U[s];
    const int F8 = (f + 7) >> 3, P8 = (p + 7) >> 3;
    const float2* L = ws + f_off[s];
    float* Tf = wt + t_off[s];
    float* Tb = wt + bwd_base + t_off[s];
    const int e = threadIdx.x >> 5, rr = threadIdx.x & 31;  // pivot in its chunk, row in the block
    const int row = bl.y * 32 + rr;
    if ((row >> 3) >= F8) return;
    const int rg = row >> 3, rl = row & 7;
    for (int kc = 0; kc < P8; ++kc) {
        const int k = kc * 8 + e;
        const float2 v = (k < p && row < f) ? L[(int64_t)k * f + row] : make_float2(0.f, 0.f);
        float* bf = Tf + ((int64_t)kc * F8 + rg) * 128;   // forward: line = row, element = pivot
        bf[swz32(rl, e)] = v.x;
        bf[64 + swz32(rl, e)] = v.y;
        float* bb = Tb + ((int64_t)rg * P8 + kc) * 128;   // backward: line = pivot, element = row
        bb[swz32(e, rl)] = v.x;
        bb[64 + swz32(e, rl)] = v.y;
    }
}

}  // namespace

// floats of one tiled copy of a front (8 x 8 blocks, two planes)
int64_t tiled_panel_floats(int p, int f) { return (int64_t)((f + 7) / 8) * ((p + 7) / 8) * 128; }

void pack_tiled(const int2* blocks, int64_t nblocks, const int64_t* f_off, const int64_t* t_off, const int32_t* P,
                const int32_t* U, const float2* ws, float* wt, int64_t bwd_base, cudaStream_t st) {
    for (int64_t b = 0; b < nblocks; b += 65535 * 64) {
        const int64_t n = std::min<int64_t>(nblocks - b, 65535 * 64);
        pack_tiled_kernel<<<(unsigned)n, 256, 0, st>>>(blocks + b, f_off, t_off, P, U, ws, wt, bwd_base);
        MWI_CHECK_LAUNCH();
    }
}

int sweep_tc_ctas() {
    static int n = 0;
    if (!n) {
        int dev = 0, sms = 0;
        MWI_CUDA(cudaGetDevice(&dev));
        MWI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        n = std::max(1, sms * kCtasPerSm);
    }
    return n;
}

template <int MODE>
static void launch_tc(const TileDesc* tiles, int64_t ntiles, int m, const int32_t* urows, const int2* asm2,
                      const float* wt, const float2* dinv, float2* Y, float2* Z, float2* upd, int* err,
                      cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        MWI_CUDA(cudaFuncSetAttribute(sweep_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kSmemBytes));
        attr = true;
    }
    const int nchunks = (m + 31) / 32;
    const int64_t total = ntiles * nchunks;
    const int grid = (int)std::min<int64_t>(total, sweep_tc_ctas());
    sweep_tc_kernel<MODE><<<grid, kThreads, kSmemBytes, st>>>(tiles, (int)ntiles, nchunks, urows, asm2, wt, dinv, Y,
                                                              Z, upd, m, err);
    MWI_CHECK_LAUNCH();
}

void sweep_tc_level(bool backward, const TileDesc* tiles, int64_t ntiles, int m, const int32_t* urows,
                    const int2* asm2, const float* wt, const float2* dinv, float2* Y, float2* Z, float2* upd,
                    int* err, cudaStream_t st) {
    if (ntiles <= 0) return;
    MWI_REQUIRE(ntiles * ((m + 31) / 32) < ((int64_t)1 << 31), MWI_EINVAL, "too many sweep tiles");
    if (backward) launch_tc<kBwdT>(tiles, ntiles, m, urows, asm2, wt, dinv, Y, Z, upd, err, st);
    else launch_tc<kFwdT>(tiles, ntiles, m, urows, asm2, wt, dinv, Y, Z, upd, err, st);
}

}  // namespace mwi
