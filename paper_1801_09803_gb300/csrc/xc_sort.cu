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
// ranks its keys with __match_any_sync and warps are ordered through shared
// counters.  A tile is 256 threads x 16 rounds = 4096 keys.
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

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin, uint64_t *kout,
                                                           uint32_t *vout, size_t n, int shift,
                                                           const uint32_t *__restrict__ offs, uint32_t n_tiles) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    run[tid] = offs[(size_t)tid * n_tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_THREADS / 32; ++w) wc[w][tid] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * RS_TILE;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * RS_THREADS + tid;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? (uint32_t)((key >> shift) & 255) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt_mask);
        int leader = 31 - __clz(peers);
        if (valid && lane == leader) wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wc[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) {
            s += wc[w][tid];
            wc[w][tid] = 0;
        }
        run[tid] += s;
        __syncthreads();
    }
}

__global__ void k_gather_lines(LinesDev L, size_t n, const uint64_t *skeys, const uint32_t *perm, double *nu,
                               float *elower, float *A, float *gref, float *nT, int16_t *g, int16_t *j) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t s = perm[i];
        nu[i] = val_of_key(skeys[i]);
        elower[i] = L.elower[s];
        A[i] = L.A[s];
        gref[i] = L.gamma_ref[s];
        nT[i] = L.n_T[s];
        g[i] = L.g_up[s];
        j[i] = L.j_lo ? L.j_lo[s] : (int16_t)0;
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
