// distance.cu -- the distance matrix and the enclosing radius.
//
// The paper takes the distance matrix D as its input (Sec. 2: D[i,j] =
// d(point i, point j), D[i,i] = 0). From points this library fixes one float32
// formula so that every diameter, and so the whole filtration order, is
// reproducible bit for bit: s = 0; s = s + (x_k - y_k)^2 for k = 0..dim-1,
// each operation rounded to nearest with no fused multiply-add, then a
// correctly rounded square root. (y - x) is the exact negation of (x - y), so
// D[i][j] and D[j][i] are computed independently yet are equal.
//
// The enclosing radius R = min_x max_y d(x, y) (Sec. "Filtering Out Simplices
// by Diameter Equal to the Enclosing Radius") bounds every nonzero interval.
#include "internal.h"

namespace rpp {

namespace {

constexpr int DT = 32;  // tile edge

// One block computes a DT x DT tile of D with 32 x 8 threads (4 rows per
// thread). The tile's row and column points are staged in shared memory.
__global__ void __launch_bounds__(256) k_distance_smem(const float *__restrict__ X, int64_t n,
                                                        int dim, float *__restrict__ D,
                                                        int64_t ld) {
    extern __shared__ float sm[];
    float *rows = sm;             // DT x dim
    float *cols = sm + DT * dim;  // DT x dim
    const int64_t r0 = (int64_t)blockIdx.y * DT, c0 = (int64_t)blockIdx.x * DT;
    const int tid = threadIdx.y * DT + threadIdx.x;
    for (int i = tid; i < DT * dim; i += 256) {
        int64_t pr = r0 + i / dim, pc = c0 + i / dim;
        rows[i] = pr < n ? X[pr * dim + i % dim] : 0.0f;
        cols[i] = pc < n ? X[pc * dim + i % dim] : 0.0f;
    }
    __syncthreads();
    const int64_t c = c0 + threadIdx.x;
    if (c >= ld) return;
    for (int rr = threadIdx.y; rr < DT; rr += 8) {
        const int64_t r = r0 + rr;
        if (r >= n) break;
        float out = 0.0f;
        if (c < n) {
            float s = 0.0f;
            const float *a = rows + rr * dim, *b = cols + threadIdx.x * dim;
            for (int k = 0; k < dim; ++k) {
                float d = __fsub_rn(a[k], b[k]);
                s = __fadd_rn(s, __fmul_rn(d, d));
            }
            out = __fsqrt_rn(s);
        }
        D[r * ld + c] = out;  // padding columns c in [n, ld) get 0 and are never read
    }
}

// Same arithmetic reading the points from global memory, for large dim.
__global__ void k_distance_global(const float *__restrict__ X, int64_t n, int dim,
                                  float *__restrict__ D, int64_t ld) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (c >= ld || r >= n) return;
    float out = 0.0f;
    if (c < n) {
        float s = 0.0f;
        for (int k = 0; k < dim; ++k) {
            float d = __fsub_rn(X[r * dim + k], X[c * dim + k]);
            s = __fadd_rn(s, __fmul_rn(d, d));
        }
        out = __fsqrt_rn(s);
    }
    D[r * ld + c] = out;
}

__global__ void k_copy_validate(const float *__restrict__ src, int64_t n, float *__restrict__ D,
                                int64_t ld, DevState *st) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    if (c >= ld || r >= n) return;
    float v = 0.0f;
    unsigned err = 0;
    if (c < n) {
        v = src[r * n + c];
        if (!isfinite(v)) err |= ERR_NONFINITE;
        else if (v < 0.0f) err |= ERR_NEGATIVE;
        if (r == c && v != 0.0f) err |= ERR_DIAGONAL;
        if (v != src[c * n + r]) err |= ERR_ASYMMETRIC;
        v = v + 0.0f;  // -0.0 becomes +0.0, so float bit patterns order diameters
    }
    D[r * ld + c] = v;
    if (err) atomicOr(&st->err, err);
}

// One warp per row: row maximum, then an atomic minimum over rows. Distances
// are non-negative, so their float bit patterns order like unsigned integers.
__global__ void k_row_max_min(const float *__restrict__ D, int64_t n, int64_t ld, DevState *st) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        float m = 0.0f;
        bool finite = true;
        for (int64_t c = lane; c < n; c += 32) {
            const float x = D[r * ld + c];
            finite &= isfinite(x);
            m = fmaxf(m, x);
        }
        if (!__all_sync(0xffffffffu, finite) && lane == 0) atomicOr(&st->err, ERR_NONFINITE);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMin((unsigned int *)&st->R, __float_as_uint(m));
    }
}

__global__ void k_init_radius(DevState *st) { st->R = __uint_as_float(0x7f800000u); }

__global__ void k_final_threshold(DevState *st, float t_user) { st->t = fminf(t_user, st->R); }

}  // namespace

void launch_distance_matrix(const float *X, int64_t n, int32_t dim, float *D, int64_t ld,
                            cudaStream_t s) {
    if (n <= 0) return;
    const size_t smem = 2ull * DT * dim * sizeof(float);
    if (smem <= 48 * 1024) {
        dim3 grid((unsigned)((ld + DT - 1) / DT), (unsigned)((n + DT - 1) / DT));
        ++g_launches;
        k_distance_smem<<<grid, dim3(DT, 8), smem, s>>>(X, n, dim, D, ld);
    } else {
        dim3 grid((unsigned)((ld + 127) / 128), (unsigned)n);
        ++g_launches;
        k_distance_global<<<grid, 128, 0, s>>>(X, n, dim, D, ld);
    }
}

void launch_copy_validate_distances(const float *src, int64_t n, float *D, int64_t ld,
                                    DevState *st, cudaStream_t s) {
    if (n <= 0) return;
    dim3 grid((unsigned)((ld + 127) / 128), (unsigned)n);
    ++g_launches;
    k_copy_validate<<<grid, 128, 0, s>>>(src, n, D, ld, st);
}

void launch_enclosing_radius(const float *D, int64_t n, int64_t ld, DevState *st, float t_user,
                             cudaStream_t s) {
    ++g_launches;
    k_init_radius<<<1, 1, 0, s>>>(st);
    if (n > 0) {
        int64_t warps = n < 152 * 32 ? n : 152 * 32;
        int blocks = (int)((warps * 32 + 255) / 256);
        ++g_launches;
        k_row_max_min<<<blocks, 256, 0, s>>>(D, n, ld, st);
    }
    ++g_launches;
    k_final_threshold<<<1, 1, 0, s>>>(st, t_user);
}

}  // namespace rpp
