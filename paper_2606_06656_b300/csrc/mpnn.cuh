// mpnn.cuh -- the learned initialiser's device structures and launchers
// (mpnn.cu), used by the C ABI layer (api.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace cls {
namespace mp {

constexpr int kHid = 64;   // hidden width
constexpr int kFv = 4;     // variable features
constexpr int kFc = 12;    // constraint features

// Device view of the incidence graph of a problem.
struct Graph {
  int n = 0, m = 0, n_free = 0;
  const int32_t* con_off = nullptr;   // m+1, literals of constraint c
  const int32_t* con_var = nullptr;   // nnz, variable of each literal
  const float* con_sgn = nullptr;     // nnz, +-1
  const int32_t* var_off = nullptr;   // n+1, rows of variable v
  const int32_t* var_con = nullptr;   // nnz, constraint of each row
  const float* var_sgn = nullptr;     // nnz, +-1
  const float* isL = nullptr;         // m, 1/sqrt(L_c)
  const float* isd = nullptr;         // n, 1/sqrt(max(deg_v, 1))
  const float* fv = nullptr;          // n x 4
  const float* fc = nullptr;          // m x 12
  const uint8_t* fixed = nullptr;     // n or null
  const float* fixed_val = nullptr;   // n or null
};

// Offsets (floats) of every tensor in the flat parameter vector.
struct ParamLayout {
  int64_t W_vin, b_vin, W_cin, b_cin, W_c[2], b_c[2], W_v[2], b_v[2], w_out, b_out, total;
};
ParamLayout param_layout();
std::vector<int32_t> fan_in_table();   // per parameter: fan-in, 0 = ReLU bias, -1 = zero

// Offsets (floats) in the activation workspace kept from forward to backward.
struct ActLayout {
  size_t hv0, hc0, ac[2], hc[2], av[2], hv[2], dhv, dhc, dA, dw_part, emb_part, emb_red,
      head_part;
  int n_dw_blk, emb_chunk, n_emb_blk;
  size_t total_floats;
};
ActLayout act_layout(int n, int m);

cudaError_t forward(const Graph& G, const float* P, float* z, float* act, cudaStream_t s);
cudaError_t points(const Graph& G, const float* z, int R, uint64_t seed, int64_t r_off, float tau,
                   float* x0, cudaStream_t s);
cudaError_t head_grad(const Graph& G, const float* z, const float* x0, const float* gx0, int R,
                      const int8_t* target, float lam, float* dz, cudaStream_t s);
cudaError_t backward(const Graph& G, const float* P, const float* dz, float* dP, float* act,
                     cudaStream_t s);
cudaError_t adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t s);
cudaError_t param_init(const int32_t* fan_in, int64_t n, uint64_t seed, float* p, cudaStream_t s);

}  // namespace mp
}  // namespace cls
