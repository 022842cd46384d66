// xc_sort.cu -- load + sort of the line list by wavenumber on the device.
//
// Keys are the float64 bit patterns of nu mapped to an order-preserving
// unsigned integer; an LSD radix sort with 8-bit digits (stable, so equal
// wavenumbers keep their input order) carries a 32-bit index payload, and a
// gather pass then reorders every field.  Digit positions where all keys share
// one digit value are skipped (decided once from a global histogram).
//
// Per pass: (1) per-tile digit histograms, (2) digit totals and exclusive scan
// into per-(digit, tile) output offsets, (3) a stable scatter where each warp
// ranks its keys with __match_any_sync, warps are ordered through shared
// counters, and each half-tile is ordered by digit in shared memory before it is
// written out.  A tile is 256 threads x 16 rounds = 4096 keys.
#include <stdio.h>

#include "xc_internal.cuh"

namespace xc {

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__device__ inline uint64_t key_of(double v) {
    uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double val_of_key(uint64_t k) {
    uint64_t b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// keys, payload and input validation; flag bit 1 = invalid value
__global__ void k_make_keys(LinesDev L, size_t n, uint64_t *keys, uint32_t *vals, int *flag) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double nu = L.nu[i];
        float e = L.elower[i], a = L.A[i], gr = L.gamma_ref[i], nt = L.n_T[i];
        int16_t g = L.g_up[i];
        bool ok = isfinite(nu) && nu > 0.0 && isfinite(e) && e >= 0.0f && isfinite(a) && a >= 0.0f &&
                  isfinite(gr) && gr >= 0.0f && isfinite(nt) && g >= 0;
        if (!ok) atomicOr(flag, 1);
        keys[i] = key_of(nu);
        vals[i] = (uint32_t)i;
    }
}

// global histogram of all 8 digit positions (for pass skipping)
__global__ void k_rs_global_hist(const uint64_t *keys, size_t n, unsigned long long *ghist /*[8][256]*/) {
    __shared__ unsigned int h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
#pragma unroll
        for (int d = 0; d < 8; ++d) atomicAdd(&h[d][(k >> (8 * d)) & 255], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
        unsigned int v = (&h[0][0])[i];
        if (v) atomicAdd(&ghist[i], (unsigned long long)v);
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_tile_hist(const uint64_t *keys, size_t n, int shift,
                                                             uint32_t *hist, uint32_t n_tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// one CTA per digit: total of its row
__global__ void k_rs_row_total(const uint32_t *hist, uint32_t n_tiles, uint32_t *tot) {
    __shared__ uint32_t s[256];
    uint32_t acc = 0;
    const uint32_t *row = hist + (size_t)blockIdx.x * n_tiles;
    for (uint32_t t = threadIdx.x; t < n_tiles; t += 256) acc += row[t];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = s[0];
}

// one CTA per digit: row offsets = digit base + exclusive prefix over tiles
__global__ void k_rs_row_scan(uint32_t *hist, uint32_t n_tiles, const uint32_t *tot) {
    __shared__ uint32_t s[256];
    __shared__ uint32_t base;
    if (threadIdx.x == 0) {
        uint32_t b = 0;
        for (uint32_t d = 0; d < blockIdx.x; ++d) b += tot[d];
        base = b;
    }
    __syncthreads();
    uint32_t carry = base;
    uint32_t *row = hist + (size_t)blockIdx.x * n_tiles;
    for (uint32_t t0 = 0; t0 < n_tiles; t0 += 256) {
        uint32_t t = t0 + threadIdx.x;
        uint32_t v = t < n_tiles ? row[t] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {  // Hillis-Steele inclusive scan
            uint32_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (t < n_tiles) row[t] = carry + s[threadIdx.x] - v;
        uint32_t chunk = s[255];
        __syncthreads();
        carry += chunk;
    }
}

// Stable scatter of one tile, in two halves of RS_HALF keys.  Each half is ranked in
// shared memory first (digit counts, their exclusive scan, then per round the warp ranks of
// __match_any_sync and the counts of earlier warps, as a stable sort by digit), and then
// written out in that order: consecutive threads write consecutive positions of a digit's
// run, instead of every key going to its own scattered address.  The global position of a
// key is the tile's offset for its digit plus its stable rank among the tile's keys of that
// digit, so the output is that of a stable LSD pass.
constexpr int RS_HALF_ROUNDS = RS_ROUNDS / 2;
constexpr int RS_HALF = RS_THREADS * RS_HALF_ROUNDS;
static_assert(RS_THREADS == 256, "one thread per digit value in the per-digit tables");

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin, uint64_t *kout,
                                                           uint32_t *vout, size_t n, int shift,
                                                           const uint32_t *__restrict__ offs, uint32_t n_tiles) {
    __shared__ uint64_t skey[RS_HALF];
    __shared__ uint32_t sval[RS_HALF];
    __shared__ uint32_t wc[RS_THREADS / 32][256];   // per round: keys of each digit per warp
    __shared__ uint32_t grun[256];                  // next global position per digit
    __shared__ uint32_t sstart[256];                // first local position per digit (this half)
    __shared__ uint32_t slrun[256];                 // next local position per digit
    __shared__ uint32_t scnt[256];                  // keys per digit (this half)
    __shared__ uint32_t swt[RS_THREADS / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    grun[tid] = offs[(size_t)tid * n_tiles + blockIdx.x];
    scnt[tid] = 0;
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) wc[w][tid] = 0;
    const size_t tbase = (size_t)blockIdx.x * RS_TILE;
    for (int half = 0; half < 2; ++half) {
        const size_t base = tbase + (size_t)half * RS_HALF;
        uint64_t key[RS_HALF_ROUNDS];
        uint32_t val[RS_HALF_ROUNDS], dig[RS_HALF_ROUNDS];
#pragma unroll
        for (int r = 0; r < RS_HALF_ROUNDS; ++r) {
            const size_t i = base + (size_t)r * RS_THREADS + tid;
            const bool valid = i < n;
            key[r] = valid ? kin[i] : 0ull;
            val[r] = valid ? vin[i] : 0u;
            dig[r] = valid ? (uint32_t)((key[r] >> shift) & 255) : 256u;
        }
        __syncthreads();   // the previous half's tables are no longer read
        // digit counts of the half (one shared atomic per distinct digit of a warp)
#pragma unroll
        for (int r = 0; r < RS_HALF_ROUNDS; ++r) {
            const unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
            if (dig[r] < 256u && lane == 31 - __clz(peers)) atomicAdd(&scnt[dig[r]], (uint32_t)__popc(peers));
        }
        __syncthreads();
        // exclusive scan of the counts over the 256 digits
        {
            const uint32_t v = scnt[tid];
            uint32_t inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            if (lane == 31) swt[warp] = inc;
            __syncthreads();
            uint32_t wpre = 0;
#pragma unroll
            for (int w = 0; w < RS_THREADS / 32; ++w) wpre += w < warp ? swt[w] : 0u;
            sstart[tid] = slrun[tid] = wpre + inc - v;
        }
        __syncthreads();
        // stable local ranks, round by round, into shared memory
#pragma unroll
        for (int r = 0; r < RS_HALF_ROUNDS; ++r) {
            const uint32_t d = dig[r];
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && lane == 31 - __clz(peers)) wc[warp][d] = __popc(peers);
            __syncthreads();
            if (d < 256u) {
                uint32_t pos = slrun[d] + __popc(peers & lt_mask);
                for (int w = 0; w < warp; ++w) pos += wc[w][d];
                skey[pos] = key[r];
                sval[pos] = val[r];
            }
            __syncthreads();
            uint32_t add = 0;
#pragma unroll
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                add += wc[w][tid];
                wc[w][tid] = 0;
            }
            slrun[tid] += add;
            __syncthreads();   // counters reset and advanced before the next round uses them
        }
        // write the half out in local order: runs of one digit go to consecutive addresses
        const uint32_t nvalid = slrun[255];   // every valid key of the half has been placed
#pragma unroll
        for (int r = 0; r < RS_HALF_ROUNDS; ++r) {
            const uint32_t idx = (uint32_t)(r * RS_THREADS + tid);
            if (idx < nvalid) {
                const uint64_t k = skey[idx];
                const uint32_t d = (uint32_t)((k >> shift) & 255);
                const uint32_t gpos = grun[d] + (idx - sstart[d]);
                kout[gpos] = k;
                vout[gpos] = sval[idx];
            }
        }
        __syncthreads();
        grun[tid] += scnt[tid];
        scnt[tid] = 0;
    }
}

// Reorders every field by the sorted permutation.  The reads are random (one sector per
// field and line), so each thread issues the loads of GL_UNROLL lines before any store to
// keep more of them in flight.
constexpr int GL_UNROLL = 4;
__global__ void k_gather_lines(LinesDev L, size_t n, const uint64_t *__restrict__ skeys,
                               const uint32_t *__restrict__ perm, double *__restrict__ nu,
                               float *__restrict__ elower, float *__restrict__ A, float *__restrict__ gref,
                               float *__restrict__ nT, int16_t *__restrict__ g, int16_t *__restrict__ j) {
    const float *__restrict__ iE = L.elower;
    const float *__restrict__ iA = L.A;
    const float *__restrict__ iG = L.gamma_ref;
    const float *__restrict__ iN = L.n_T;
    const int16_t *__restrict__ iU = L.g_up;
    const int16_t *__restrict__ iJ = L.j_lo;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * GL_UNROLL) {
        uint32_t sidx[GL_UNROLL];
        float e[GL_UNROLL], a[GL_UNROLL], gr[GL_UNROLL], nt[GL_UNROLL];
        int16_t gu[GL_UNROLL], jl[GL_UNROLL];
        uint64_t k[GL_UNROLL];
#pragma unroll
        for (int u = 0; u < GL_UNROLL; ++u) {
            const size_t i = i0 + (size_t)u * stride;
            sidx[u] = i < n ? perm[i] : 0u;
            k[u] = i < n ? skeys[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < GL_UNROLL; ++u) {
            const size_t i = i0 + (size_t)u * stride;
            if (i < n) {
                const uint32_t s = sidx[u];
                e[u] = iE[s];
                a[u] = iA[s];
                gr[u] = iG[s];
                nt[u] = iN[s];
                gu[u] = iU[s];
                jl[u] = iJ ? iJ[s] : (int16_t)0;
            }
        }
#pragma unroll
        for (int u = 0; u < GL_UNROLL; ++u) {
            const size_t i = i0 + (size_t)u * stride;
            if (i < n) {
                nu[i] = val_of_key(k[u]);
                elower[i] = e[u];
                A[i] = a[u];
                gref[i] = gr[u];
                nT[i] = nt[u];
                g[i] = gu[u];
                j[i] = jl[u];
            }
        }
    }
}

// already-sorted input: copy, identity permutation, order check (flag bit 2)
__global__ void k_copy_sorted(LinesDev L, size_t n, double *nu, float *elower, float *A, float *gref, float *nT,
                              int16_t *g, int16_t *j, uint32_t *perm, int *flag) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = L.nu[i];
        if (i + 1 < n && !(v <= L.nu[i + 1])) atomicOr(flag, 2);
        nu[i] = v;
        elower[i] = L.elower[i];
        A[i] = L.A[i];
        gref[i] = L.gamma_ref[i];
        nT[i] = L.n_T[i];
        g[i] = L.g_up[i];
        j[i] = L.j_lo ? L.j_lo[i] : (int16_t)0;
        perm[i] = (uint32_t)i;
    }
}

static unsigned grid_for(size_t n, unsigned per_sm = 8) {
    size_t b = (n + 255) / 256;
    size_t cap = (size_t)152 * per_sm;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_sort_lines(const LinesDev &in, size_t n, bool assume_sorted, DevBuf *tmp, double *nu,
                              float *elower, float *A, float *gref, float *nT, int16_t *g, int16_t *j,
                              uint32_t *perm, int *d_flag, cudaStream_t s, cudaEvent_t *ev, int64_t *launches,
                              bool *bad_input, bool *unsorted) {
    cudaError_t e;
    *bad_input = false;
    *unsorted = false;
    if ((e = cudaMemsetAsync(d_flag, 0, sizeof(int), s)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    if (assume_sorted) {
        k_copy_sorted<<<grid_for(n), 256, 0, s>>>(in, n, nu, elower, A, gref, nT, g, j, perm, d_flag);
        ++*launches;
        // validation of values shares k_make_keys' checks: run it into scratch keys
        if ((e = tmp[0].ensure(n * 8 + 16)) != cudaSuccess) return e;
        if ((e = tmp[1].ensure(n * 4 + 16)) != cudaSuccess) return e;
        k_make_keys<<<grid_for(n), 256, 0, s>>>(in, n, tmp[0].as<uint64_t>(), tmp[1].as<uint32_t>(), d_flag);
        ++*launches;
        if (ev) {
            cudaEventRecord(ev[1], s);
            cudaEventRecord(ev[2], s);
        }
    } else {
        const uint32_t n_tiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
        // scratch: keys x2 (8 B), vals x2 (4 B), tile hist (256 x n_tiles), totals, global hist
        if ((e = tmp[0].ensure(n * 8 + 16)) != cudaSuccess) return e;
        if ((e = tmp[1].ensure(n * 8 + 16)) != cudaSuccess) return e;
        if ((e = tmp[2].ensure(n * 4 + 16)) != cudaSuccess) return e;
        if ((e = tmp[3].ensure(n * 4 + 16)) != cudaSuccess) return e;
        if ((e = tmp[4].ensure((size_t)256 * n_tiles * 4 + 256 * 4 + 8 * 256 * 8 + 64)) != cudaSuccess) return e;
        uint64_t *k0 = tmp[0].as<uint64_t>(), *k1 = tmp[1].as<uint64_t>();
        uint32_t *v0 = tmp[2].as<uint32_t>(), *v1 = tmp[3].as<uint32_t>();
        uint32_t *hist = tmp[4].as<uint32_t>();
        uint32_t *tot = hist + (size_t)256 * n_tiles;
        unsigned long long *ghist = reinterpret_cast<unsigned long long *>(tot + 256 + 8);  // 16-byte aligned
        ghist = reinterpret_cast<unsigned long long *>((reinterpret_cast<uintptr_t>(ghist) + 15) & ~uintptr_t(15));
        k_make_keys<<<grid_for(n), 256, 0, s>>>(in, n, k0, v0, d_flag);
        if ((e = cudaMemsetAsync(ghist, 0, 8 * 256 * 8, s)) != cudaSuccess) return e;
        k_rs_global_hist<<<grid_for(n, 4), 256, 0, s>>>(k0, n, ghist);
        *launches += 2;
        unsigned long long h_g[8 * 256];
        if ((e = cudaMemcpyAsync(h_g, ghist, sizeof(h_g), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        for (int d = 0; d < 8; ++d) {
            bool trivial = false;
            for (int b = 0; b < 256; ++b)
                if (h_g[d * 256 + b] == (unsigned long long)n) trivial = true;
            if (trivial) continue;
            int shift = 8 * d;
            k_rs_tile_hist<<<n_tiles, RS_THREADS, 0, s>>>(k0, n, shift, hist, n_tiles);
            k_rs_row_total<<<256, 256, 0, s>>>(hist, n_tiles, tot);
            k_rs_row_scan<<<256, 256, 0, s>>>(hist, n_tiles, tot);
            k_rs_scatter<<<n_tiles, RS_THREADS, 0, s>>>(k0, v0, k1, v1, n, shift, hist, n_tiles);
            *launches += 4;
            uint64_t *tk = k0; k0 = k1; k1 = tk;
            uint32_t *tv = v0; v0 = v1; v1 = tv;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[1], s);
        if ((e = cudaMemcpyAsync(perm, v0, n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
        k_gather_lines<<<grid_for(n), 256, 0, s>>>(in, n, k0, v0, nu, elower, A, gref, nT, g, j);
        ++*launches;
        if (ev) cudaEventRecord(ev[2], s);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int h_flag = 0;
    if ((e = cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *bad_input = (h_flag & 1) != 0;
    *unsorted = (h_flag & 2) != 0;
    return cudaSuccess;
}

}  // namespace xc
