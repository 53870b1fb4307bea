// Device state and launchers of the learned-initial-guess network (net.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace stmg {

constexpr int kNetMaxLayers = 8;

struct NetDev {
  int L = 0;                       // number of convolution layers
  int nt = 1;                      // time DoFs per slab (input has 2 nt channels, output nt)
  int nx = 0, ny = 0, nz = 1;      // node grid
  int64_t V = 0;
  // activations live on the node grid padded by one zero layer on every side (nx+2, ny+2, nz+2),
  // so that every 3x3x3 neighbour of a grid node is a row of the same matrix; the halo stays zero
  int nxp = 0, nyp = 0, nzp = 0;
  int64_t Vp = 0;
  int ch[kNetMaxLayers + 1] = {};  // true channel counts
  int cp[kNetMaxLayers + 1] = {};  // padded channel counts (16 or 64)
  float su = 1.f, sf = 1.f, so = 1.f;  // input / output scalings
  int step = 0;                    // Adam step counter
  // parameters: FP32 masters [27][cp_out][cp_in], BF16 forward and transposed copies, biases
  float* w32[kNetMaxLayers] = {};
  __nv_bfloat16* wt[kNetMaxLayers] = {};
  __nv_bfloat16* wtT[kNetMaxLayers] = {};
  float* bias[kNetMaxLayers] = {};
  float *gw[kNetMaxLayers] = {}, *gb[kNetMaxLayers] = {};
  float *mw[kNetMaxLayers] = {}, *vw[kNetMaxLayers] = {}, *mb[kNetMaxLayers] = {}, *vb[kNetMaxLayers] = {};
  // activations act[0..L-1] ([V][cp[l]]), output (FP32 [V][cp[L]]), gradients grad[1..L]
  __nv_bfloat16* act[kNetMaxLayers + 1] = {};
  float* out = nullptr;
  __nv_bfloat16* grad[kNetMaxLayers + 1] = {};
  double* loss = nullptr;          // device scalar
  // tensor maps of the tensor-core convolutions: forward (input act[l], weights wt[l]) and backward
  // data (input grad[l+1], weights wtT[l]) of every layer
  CUtensorMap tm_in_f[kNetMaxLayers], tm_w_f[kNetMaxLayers], tm_in_b[kNetMaxLayers], tm_w_b[kNetMaxLayers];
  int* status = nullptr;           // device status word of the bounded waits (the context's)
};

// row of node v (lexicographic on the nx x ny x nz grid) in the padded activation matrices
inline int64_t net_row(const NetDev& n, int64_t v) {
  const int64_t x = v % n.nx, y = (v / n.nx) % n.ny, z = v / ((int64_t)n.nx * n.ny);
  return (x + 1) + (int64_t)n.nxp * ((y + 1) + (int64_t)n.nyp * (z + 1));
}

int net_pad(int c);
cudaError_t net_make_tmaps(NetDev& n);
cudaError_t net_forward(const NetDev& n, const double* u_prev, const double* f, cudaStream_t s);
cudaError_t net_guess(const NetDev& n, const double* u_prev, double* guess, cudaStream_t s);
cudaError_t net_backward(NetDev& n, const double* u_prev, const double* u_target, double* loss, cudaStream_t s);
cudaError_t net_adam(NetDev& n, float lr, cudaStream_t s);
cudaError_t net_refresh_bf16(NetDev& n, cudaStream_t s);

}  // namespace stmg
