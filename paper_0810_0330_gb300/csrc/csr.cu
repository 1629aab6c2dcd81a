// csr.cu -- y = A x for a real CSR matrix on sm_103a (FP64, and the FP32 copy
// of the mixed-precision path).
//
// The paper's first test matrices (Sec. 2, 3) are sparse SPD matrices with a
// handful of entries per row, so by default one thread owns one row and walks
// it in order.  Rows with more entries read their values and column indices
// better with a group of 2, 4 or 8 lanes per row (consecutive lanes read
// consecutive entries; the group's partial sums are combined by shuffles in a
// fixed order).  Which shape is fastest depends on the matrix and on the GPU:
// the context's autotuner (seed_params.autotune) times the shapes in
// kCsrShape on the matrix itself and keeps the best.  Every shape has a fixed
// summation order, so results are reproducible for a given shape.  Several
// right-hand sides are handled by grid.y; columns whose flag in col_active is
// 0 are skipped (finished CG systems).
#include "device_common.cuh"
#include "seed_internal.h"

namespace seedk {

template <class R>
__global__ void __launch_bounds__(256) k_csr_spmv(CsrOpT<R> op, const R *__restrict__ in, int64_t ldi,
                                                  R *__restrict__ out, int64_t ldo,
                                                  const int32_t *__restrict__ col_active) {
  const int col = blockIdx.y;
  if (col_active != nullptr && col_active[col] == 0) return;
  in += (int64_t)col * ldi;
  out += (int64_t)col * ldo;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < op.n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = __ldg(op.row_ptr + r), e = __ldg(op.row_ptr + r + 1);
    R s = 0;
    for (int32_t k = b; k < e; ++k) s = fma(__ldg(op.vals + k), __ldg(in + __ldg(op.col_idx + k)), s);
    out[r] = s;
  }
}

// TPR lanes per row.  The row loop is warp-uniform (every lane of a warp runs
// the same number of trips) so that the shuffles see the whole warp.
template <class R, int TPR>
__global__ void __launch_bounds__(512) k_csr_spmv_group(CsrOpT<R> op, const R *__restrict__ in, int64_t ldi,
                                                        R *__restrict__ out, int64_t ldo,
                                                        const int32_t *__restrict__ col_active) {
  const int col = blockIdx.y;
  if (col_active != nullptr && col_active[col] == 0) return;
  in += (int64_t)col * ldi;
  out += (int64_t)col * ldo;
  const int g = threadIdx.x & (TPR - 1);
  const int64_t rows_per_block = blockDim.x / TPR;
  const int64_t stride = (int64_t)gridDim.x * rows_per_block;
  const int64_t warp_first = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / TPR;
  for (int64_t base = warp_first; base < op.n; base += stride) {
    const int64_t r = base + (threadIdx.x & 31) / TPR;
    R s = 0;
    if (r < op.n) {
      const int32_t b = __ldg(op.row_ptr + r), e = __ldg(op.row_ptr + r + 1);
      for (int32_t k = b + g; k < e; k += TPR) s = fma(__ldg(op.vals + k), __ldg(in + __ldg(op.col_idx + k)), s);
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, TPR);
    if (g == 0 && r < op.n) out[r] = s;
  }
}

const int32_t kCsrShape[kCsrShapes][2] = {{1, 256}, {1, 128}, {1, 512}, {2, 256}, {4, 256}, {8, 256}};

template <class R>
static void launch_csr(const CsrOpT<R> &op, const R *in, int64_t ldi, R *out, int64_t ldo, int ncols,
                       const int32_t *col_active, cudaStream_t s) {
  const int tpr = op.tpr, nt = op.block;
  int64_t blocks = (op.n * tpr + nt - 1) / nt;
  if (blocks > 152 * 16) blocks = 152 * 16;
  dim3 grid((unsigned)blocks, (unsigned)ncols);
  switch (tpr) {
    case 2: k_csr_spmv_group<R, 2><<<grid, nt, 0, s>>>(op, in, ldi, out, ldo, col_active); break;
    case 4: k_csr_spmv_group<R, 4><<<grid, nt, 0, s>>>(op, in, ldi, out, ldo, col_active); break;
    case 8: k_csr_spmv_group<R, 8><<<grid, nt, 0, s>>>(op, in, ldi, out, ldo, col_active); break;
    default:
      if (nt == 256) k_csr_spmv<R><<<grid, 256, 0, s>>>(op, in, ldi, out, ldo, col_active);
      else k_csr_spmv_group<R, 1><<<grid, nt, 0, s>>>(op, in, ldi, out, ldo, col_active);
  }
}

void launch_csr_spmv(const CsrOp &op, const double *in, int64_t ldi, double *out, int64_t ldo, int ncols,
                     const int32_t *col_active, cudaStream_t s) {
  launch_csr(op, in, ldi, out, ldo, ncols, col_active, s);
}

// FP32 copy of the matrix (mixed-precision path)
void launch_csr_spmv32(const CsrOp32 &op, const float *in, int64_t ldi, float *out, int64_t ldo, int ncols,
                       const int32_t *col_active, cudaStream_t s) {
  launch_csr(op, in, ldi, out, ldo, ncols, col_active, s);
}

}  // namespace seedk
