// csr.cu -- y = A x for a real CSR matrix on sm_103a (FP64).
//
// The paper's first test matrices (Sec. 2, 3) are sparse SPD matrices with a
// handful of entries per row, so one thread owns one row and walks it in
// order (a fixed summation order, identical for every launch).  Several
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

template <class R>
static void launch_csr(const CsrOpT<R> &op, const R *in, int64_t ldi, R *out, int64_t ldo, int ncols,
                       const int32_t *col_active, cudaStream_t s) {
  int64_t blocks = (op.n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  dim3 grid((unsigned)blocks, (unsigned)ncols);
  k_csr_spmv<R><<<grid, 256, 0, s>>>(op, in, ldi, out, ldo, col_active);
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
