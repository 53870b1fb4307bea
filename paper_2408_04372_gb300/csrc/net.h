// Device state and launchers of the learned-initial-guess network (net.cu).
#pragma once

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
};

int net_pad(int c);
cudaError_t net_forward(const NetDev& n, const double* u_prev, const double* f, cudaStream_t s);
cudaError_t net_guess(const NetDev& n, const double* u_prev, double* guess, cudaStream_t s);
cudaError_t net_backward(NetDev& n, const double* u_prev, const double* u_target, double* loss, cudaStream_t s);
cudaError_t net_adam(NetDev& n, float lr, cudaStream_t s);
cudaError_t net_refresh_bf16(NetDev& n, cudaStream_t s);

}  // namespace stmg
