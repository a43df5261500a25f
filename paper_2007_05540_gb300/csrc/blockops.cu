// FP64 block-product engine: lists of strided dense block products summed into output
// tiles, and block dot products.  Used by the environment update and the Rayleigh-quotient
// gradients (the block-pair contractions of Algorithm 2 with charge-matched blocks, each
// product a small dense GEMM, Section IV "list" algorithm).
#include <cuda_runtime.h>

#include <type_traits>

#include "convert.cuh"
#include "internal.h"

namespace heff {

void BList::add_block(int64_t c_off, int32_t ldc, int32_t m, int32_t n, const std::vector<BProd>& ps) {
    blocks.push_back(Block{c_off, ldc, m, n, (int32_t)block_prods.size(), (int32_t)ps.size()});
    block_prods.insert(block_prods.end(), ps.begin(), ps.end());
    for (int r0 = 0; r0 < m; r0 += tile_m)
        for (int c0 = 0; c0 < n; c0 += tile_n) {
            BTile t{};
            t.c_off = c_off + (int64_t)r0 * ldc + c0;
            t.ldc = ldc;
            t.m = m - r0 < tile_m ? m - r0 : tile_m;
            t.n = n - c0 < tile_n ? n - c0 : tile_n;
            t.prod_begin = (int32_t)prods.size();
            t.prod_count = (int32_t)ps.size();
            for (const BProd& p : ps) {
                BProd q = p;
                q.a_off += (int64_t)r0 * p.a_rs;
                q.b_off += (int64_t)c0 * p.b_cs;
                prods.push_back(q);
                flops += 2.0 * t.m * t.n * p.K;
            }
            tiles.push_back(t);
        }
}

void BList::retile(int tm, int tn) {
    std::vector<Block> bl;
    std::vector<BProd> bp;
    bl.swap(blocks);
    bp.swap(block_prods);
    tiles.clear();
    prods.clear();
    flops = 0;
    tile_m = tm;
    tile_n = tn;
    for (const Block& k : bl)
        add_block(k.c_off, k.ldc, k.m, k.n,
                  std::vector<BProd>(bp.begin() + k.prod_begin, bp.begin() + k.prod_begin + k.prod_count));
}

int blist_upload(BList& b) {
    b.d_tiles = nullptr;
    b.d_prods = nullptr;
    if (!b.tiles.empty()) {
        if (cudaMalloc((void**)&b.d_tiles, b.tiles.size() * sizeof(BTile)) != cudaSuccess ||
            cudaMemcpy(b.d_tiles, b.tiles.data(), b.tiles.size() * sizeof(BTile), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(HEFF_ERR_CUDA, "block tile upload failed");
    }
    if (!b.prods.empty()) {
        if (cudaMalloc((void**)&b.d_prods, b.prods.size() * sizeof(BProd)) != cudaSuccess ||
            cudaMemcpy(b.d_prods, b.prods.data(), b.prods.size() * sizeof(BProd), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(HEFF_ERR_CUDA, "block product upload failed");
    }
    return HEFF_OK;
}

void blist_free(BList& b) {
    cudaFree(b.d_tiles);
    cudaFree(b.d_prods);
    b.d_tiles = nullptr;
    b.d_prods = nullptr;
}

namespace {

// 64 x 64 output tile, 256 threads with 4 x 4 outputs each, K in steps of 16 through
// shared memory.  Loads follow whichever operand stride is unit so they coalesce.
__global__ void __launch_bounds__(256) bgemm_kernel(const BTile* __restrict__ tiles, const BProd* __restrict__ prods,
                                                    const double* __restrict__ A, const double* __restrict__ B,
                                                    double* __restrict__ C, const double* __restrict__ coef1,
                                                    const double* __restrict__ coef2, double scale,
                                                    const double* __restrict__ inv_scale, int accumulate) {
    __shared__ double As[16][64 + 1];
    if (inv_scale) scale /= inv_scale[0];
    __shared__ double Bs[16][64 + 1];
    const BTile t = tiles[blockIdx.x];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int pi = 0; pi < t.prod_count; ++pi) {
        const BProd p = prods[t.prod_begin + pi];
        const double coef = (p.c1 < 0 ? 1.0 : coef1[p.c1]) * (p.c2 < 0 ? 1.0 : coef2[p.c2]);
        for (int k0 = 0; k0 < p.K; k0 += 16) {
            for (int l = 0; l < 4; ++l) {
                const int idx = tid + 256 * l;
                // A: (row, kk); unit stride along k -> kk fastest, else rows fastest
                int row, kk;
                if (p.a_cs == 1) { row = idx >> 4; kk = idx & 15; } else { row = idx & 63; kk = idx >> 6; }
                As[kk][row] = (row < t.m && k0 + kk < p.K)
                                  ? coef * A[p.a_off + (int64_t)row * p.a_rs + (int64_t)(k0 + kk) * p.a_cs] : 0.0;
                int col, kb;
                if (p.b_cs == 1) { col = idx & 63; kb = idx >> 6; } else { col = idx >> 4; kb = idx & 15; }
                Bs[kb][col] = (col < t.n && k0 + kb < p.K)
                                  ? B[p.b_off + (int64_t)(k0 + kb) * p.b_rs + (int64_t)col * p.b_cs] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { a[i] = As[k][ty * 4 + i]; b[i] = Bs[k][tx * 4 + i]; }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    for (int i = 0; i < 4; ++i) {
        const int r = ty * 4 + i;
        if (r >= t.m) continue;
        for (int j = 0; j < 4; ++j) {
            const int c = tx * 4 + j;
            if (c >= t.n) continue;
            double* cp = C + t.c_off + (int64_t)r * t.ldc + c;
            *cp = accumulate ? *cp + scale * acc[i][j] : scale * acc[i][j];
        }
    }
}

// one CTA per dot: partial[d] = <X[x_off..], Y[y_off..]>, accumulated in the element type
// (FP32 vectors come from the tensor-core products, whose values carry ~1e-5 anyway)
template <typename T>
__global__ void __launch_bounds__(256) block_dot_kernel(const BDot* __restrict__ dots, const T* __restrict__ X,
                                                        const T* __restrict__ Y, double* __restrict__ partial) {
    __shared__ T sh[8];
    const BDot d = dots[blockIdx.x];
    T a = 0;
    for (int64_t i = threadIdx.x; i < d.len; i += blockDim.x) a = fma(X[d.x_off + i], Y[d.y_off + i], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        T s = 0;
        for (int w = 0; w < 8; ++w) s += sh[w];
        if constexpr (std::is_same<T, double>::value) partial[blockIdx.x] = s;
        else partial[blockIdx.x] = f32_to_f64(s);
    }
}

// out[j] = scale * sum of partial[d] for d in [off[j], off[j+1]) (dots sorted by output;
// fixed order, deterministic)
__global__ void gather_dots_kernel(const int32_t* __restrict__ off, const double* __restrict__ partial,
                                   double* __restrict__ out, int nout, double scale, int accumulate) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nout; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int d = off[j]; d < off[j + 1]; ++d) s += partial[d];
        out[j] = accumulate ? out[j] + scale * s : scale * s;
    }
}

}  // namespace

int launch_bgemm(const BList& b, const double* A, const double* B, double* C, const double* coef1,
                 const double* coef2, double scale, void* stream, const double* inv_scale) {
    if (b.tiles.empty()) return HEFF_OK;
    bgemm_kernel<<<(unsigned)b.tiles.size(), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        b.d_tiles, b.d_prods, A, B, C, coef1, coef2, scale, inv_scale, b.accumulate ? 1 : 0);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "bgemm launch: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

template <typename T>
static int block_dots_t(const BDot* d_dots, int ndots, const int32_t* d_off, const T* X, const T* Y, double* out,
                        int nout, double* scratch, double scale, void* stream, bool accumulate) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ndots > 0) {
        block_dot_kernel<T><<<ndots, 256, 0, st>>>(d_dots, X, Y, scratch);
        count_launches(1);
    }
    gather_dots_kernel<<<(nout + 255) / 256, 256, 0, st>>>(d_off, scratch, out, nout, scale, accumulate ? 1 : 0);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "block dots launch: %s", cudaGetErrorString(e));
    return HEFF_OK;
}

int launch_block_dots(const BDot* d_dots, int ndots, const int32_t* d_off, const double* X, const double* Y,
                      double* out, int nout, double* scratch, double scale, void* stream, bool accumulate) {
    return block_dots_t(d_dots, ndots, d_off, X, Y, out, nout, scratch, scale, stream, accumulate);
}

int launch_block_dots_f32(const BDot* d_dots, int ndots, const int32_t* d_off, const float* X, const float* Y,
                          double* out, int nout, double* scratch, double scale, void* stream, bool accumulate) {
    return block_dots_t(d_dots, ndots, d_off, X, Y, out, nout, scratch, scale, stream, accumulate);
}

}  // namespace heff
