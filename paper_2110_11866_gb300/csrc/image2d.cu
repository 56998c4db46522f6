// Separable 2-D Gaussian filtering of an image: the rows of the image are independent 1-D signals
// and so are its columns (the paper's discussion of 2-D signals at the start of Sec. IV), so the
// filter is one batched 1-D transform over the rows, a transpose, one batched 1-D transform over
// the columns and a transpose back. The 1-D transforms are ordinary MORLET_GAUSS plans.
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/morlet_sft.h"

namespace {

constexpr int TT = 32;  // transpose tile edge
constexpr int TR = 8;   // rows of threads per tile

// out[c][r] = in[r][c] for an rows x cols row-major array; 32 x 32 tiles through shared memory
// (padded rows: conflict-free reads and writes), every access bounds-checked.
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t rows, int64_t cols) {
  __shared__ T tile[TT][TT + 1];
  const int64_t c0 = (int64_t)blockIdx.x * TT, r0 = (int64_t)blockIdx.y * TT;
  for (int i = threadIdx.y; i < TT; i += TR) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < TT; i += TR) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;  // output row c, column r
    if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][i];
  }
}

cudaError_t transpose(const void* in, void* out, int64_t rows, int64_t cols, int elem, cudaStream_t st) {
  const int64_t gy = (rows + TT - 1) / TT;
  if (gy > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((cols + TT - 1) / TT), (unsigned)gy), block(TT, TR);
  if (elem == 8)
    transpose_kernel<double><<<grid, block, 0, st>>>(static_cast<const double*>(in), static_cast<double*>(out), rows, cols);
  else
    transpose_kernel<float><<<grid, block, 0, st>>>(static_cast<const float*>(in), static_cast<float*>(out), rows, cols);
  return cudaGetLastError();
}

struct Filter2D {
  morlet_plan_t rows = nullptr;  // ny signals of nx samples, derivative along x
  morlet_plan_t cols = nullptr;  // nx signals of ny samples, derivative along y
  void* work = nullptr;          // 2 ny nx elements
};

int make_plan(int64_t n_signals, int64_t len, double sigma, int32_t P, int32_t deriv, int32_t precision,
              void* stream, morlet_plan_t* out) {
  std::vector<int64_t> lens((size_t)n_signals, len);
  morlet_plan_desc d{};
  d.n_signals = n_signals;
  d.lengths = lens.data();
  d.n_scales = 1;
  d.sigmas = &sigma;
  d.K = P + 1;
  d.method = MORLET_GAUSS;
  d.transform = MORLET_SFT;
  d.precision = precision;
  d.deriv = deriv;
  d.flags = MORLET_FLAG_AUTOTUNE;  // the schedule timed once per image shape, when the plans are made
  return morlet_plan(out, &d, stream);
}

}  // namespace

extern "C" int gauss_filter_2d(const void* img, int64_t ny, int64_t nx, double sigma, int32_t P, int32_t deriv_y,
                               int32_t deriv_x, int32_t precision, void* out, void* stream) {
  if (!img || !out || ny < 1 || nx < 1 || P < 0 || deriv_y < 0 || deriv_y > 2 || deriv_x < 0 || deriv_x > 2)
    return MORLET_ERR_ARG;
  if (precision < MORLET_FP32_PLAIN || precision > MORLET_FP64) return MORLET_ERR_ARG;
  if ((ny + TT - 1) / TT > 65535 || (nx + TT - 1) / TT > 65535) return MORLET_ERR_ARG;
  // The two plans and the workspace are cached per key; the cache lives until process exit.
  static std::mutex mu;
  static std::map<std::tuple<int, int64_t, int64_t, double, int, int, int, int>, Filter2D> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MORLET_ERR_CUDA;
  const int elem = precision == MORLET_FP64 ? 8 : 4;
  Filter2D f;
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, ny, nx, sigma, (int)P, (int)deriv_y, (int)deriv_x, (int)precision);
    auto it = cache.find(key);
    if (it != cache.end()) {
      f = it->second;
    } else {
      int rc = make_plan(ny, nx, sigma, P, deriv_x, precision, stream, &f.rows);
      if (rc == MORLET_OK) rc = make_plan(nx, ny, sigma, P, deriv_y, precision, stream, &f.cols);
      if (rc == MORLET_OK && cudaMalloc(&f.work, (size_t)2 * ny * nx * elem) != cudaSuccess) {
        cudaGetLastError();
        rc = MORLET_ERR_NOMEM;
      }
      if (rc != MORLET_OK) {
        morlet_plan_destroy(f.rows);
        morlet_plan_destroy(f.cols);
        return rc;
      }
      cache[key] = f;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* a = static_cast<char*>(f.work);
  char* b = a + (size_t)ny * nx * elem;
  int rc = morlet_forward(f.rows, img, a, stream);  // [ny][nx]: filtered along x
  if (rc) return rc;
  if (transpose(a, b, ny, nx, elem, st) != cudaSuccess) return MORLET_ERR_CUDA;  // [nx][ny]
  rc = morlet_forward(f.cols, b, a, stream);  // [nx][ny]: filtered along y
  if (rc) return rc;
  if (transpose(a, out, nx, ny, elem, st) != cudaSuccess) return MORLET_ERR_CUDA;  // [ny][nx]
  return MORLET_OK;
}
