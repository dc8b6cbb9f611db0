// k_edges.cu -- the edge image of Sec. 3.1.
//
// One thread per pixel, one CTA per 32x8 tile.
// edges_direct_kernel (SSAO, SSGI): each lane reads its pixel and its 4 neighbours
//   straight from global memory; the neighbours' lines are the block's own rows, so
//   they are L1 hits and DRAM sees each G-buffer texel about once.
// edges_kernel (soft shadows): the tile and a one-pixel halo of depth, normals and the
//   one-sample hard shadow of Sec. 3.1 are staged in shared memory, so each staged
//   texel's hard shadow (a reconstruction, a light-space projection and a shadow-map
//   read) is computed once, not once per neighbour test.
#include "mrr_internal.cuh"
#include "shade_common.cuh"

namespace mrr {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int SX = TX + 2, SY = TY + 2;

template <typename NT, typename SMT>
__global__ void __launch_bounds__(TX* TY) edges_kernel(EdgeParams p, const float* __restrict__ depth,
                                                        const NT* __restrict__ normal,
                                                        const SMT* __restrict__ smap, uint8_t* __restrict__ E) {
  __shared__ float sd[SY][SX];
  __shared__ float snx[SY][SX], sny[SY][SX], snz[SY][SX];
  __shared__ uint8_t shs[SY][SX];
  const int W = p.v.W, H = p.v.H;
  const int x0 = blockIdx.x * TX - 1, y0 = blockIdx.y * TY - 1;
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (int k = tid; k < SX * SY; k += TX * TY) {
    const int ly = k / SX, lx = k - ly * SX;
    const int x = x0 + lx, y = y0 + ly;
    float d = -1.0f;  // outside the image
    float3 n = make_float3(0.f, 0.f, 0.f);
    uint8_t hs = 1;
    if (x >= 0 && x < W && y >= 0 && y < H) {
      const size_t i = (size_t)y * W + x;
      d = __ldg(depth + i);
      n = load_normal(normal, i);
      if (p.ssm && d < p.v.farp) hs = (uint8_t)hard_shadow(p.v, p.L, p.shadow_bias, smap, x, y, d);
    }
    sd[ly][lx] = d;
    snx[ly][lx] = n.x;
    sny[ly][lx] = n.y;
    snz[ly][lx] = n.z;
    shs[ly][lx] = hs;
  }
  __syncthreads();
  const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
  if (x >= W || y >= H) return;
  const int lx = threadIdx.x + 1, ly = threadIdx.y + 1;
  const float d = sd[ly][lx];
  uint8_t e = 0;
  if (d < p.v.farp) {
    const int ox[4] = {-1, 1, 0, 0}, oy[4] = {0, 0, -1, 1};
    const float nx = snx[ly][lx], ny = sny[ly][lx], nz = snz[ly][lx];
    const uint8_t hs = shs[ly][lx];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float dn = sd[ly + oy[k]][lx + ox[k]];
      if (dn < 0.0f) continue;          // outside the image
      if (dn >= p.v.farp) {             // sky neighbour
        e = 1;
        continue;
      }
      const float dot = nx * snx[ly + oy[k]][lx + ox[k]] + ny * sny[ly + oy[k]][lx + ox[k]] +
                        nz * snz[ly + oy[k]][lx + ox[k]];
      if (dot < p.normal_cos) e = 1;
      if (p.ssm && shs[ly + oy[k]][lx + ox[k]] != hs) e = 1;
    }
    if (x > 0 && x < W - 1) {
      const float lap = (sd[ly][lx - 1] + sd[ly][lx + 1]) - 2.0f * d;
      if (fabsf(lap) > p.depth_rel * d) e = 1;
    }
    if (y > 0 && y < H - 1) {
      const float lap = (sd[ly - 1][lx] + sd[ly + 1][lx]) - 2.0f * d;
      if (fabsf(lap) > p.depth_rel * d) e = 1;
    }
  }
  E[(size_t)y * W + x] = e;
}

// edges_direct_kernel: a lane owns a column of ER vertically adjacent pixels.  Every
// load it needs -- the column rows y0-1 .. y0+ER and the left/right neighbours of its
// pixels, at clamped addresses -- is issued before any of them is used, so a warp waits
// for memory once, and the column values double as up/down neighbours.
constexpr int ER = 2;

template <typename NT>
__global__ void __launch_bounds__(TX* TY) edges_direct_kernel(EdgeParams p, const float* __restrict__ depth,
                                                               const NT* __restrict__ normal,
                                                               uint8_t* __restrict__ E) {
  const int W = p.v.W, H = p.v.H;
  const int x = blockIdx.x * TX + threadIdx.x;
  const int y0 = (blockIdx.y * TY + threadIdx.y) * ER;
  if (x >= W || y0 >= H) return;
  const float farp = p.v.farp;
  const int xl = max(x - 1, 0), xr = min(x + 1, W - 1);
  float dc[ER + 2], dl[ER], dr[ER];
  float3 nc[ER + 2], nl[ER], nr[ER];
#pragma unroll
  for (int r = -1; r <= ER; ++r) {
    const int y = min(max(y0 + r, 0), H - 1);
    dc[r + 1] = __ldg(depth + y * W + x);
    nc[r + 1] = load_normal(normal, y * W + x);
  }
#pragma unroll
  for (int r = 0; r < ER; ++r) {
    const int y = min(y0 + r, H - 1);
    dl[r] = __ldg(depth + y * W + xl);
    dr[r] = __ldg(depth + y * W + xr);
    nl[r] = load_normal(normal, y * W + xl);
    nr[r] = load_normal(normal, y * W + xr);
  }
#pragma unroll
  for (int r = 0; r < ER; ++r) {
    const int y = y0 + r;
    if (y >= H) break;
    const float d = dc[r + 1];
    uint8_t e = 0;
    if (d < farp) {
      const float3 n = nc[r + 1];
      const bool has[4] = {x > 0, x < W - 1, y > 0, y < H - 1};
      const float dn[4] = {dl[r], dr[r], dc[r], dc[r + 2]};
      const float3 nn[4] = {nl[r], nr[r], nc[r], nc[r + 2]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!has[k]) continue;
        if (dn[k] >= farp) {  // sky neighbour
          e = 1;
          continue;
        }
        if (n.x * nn[k].x + n.y * nn[k].y + n.z * nn[k].z < p.normal_cos) e = 1;
      }
      if (has[0] && has[1]) {
        const float lap = (dn[0] + dn[1]) - 2.0f * d;
        if (fabsf(lap) > p.depth_rel * d) e = 1;
      }
      if (has[2] && has[3]) {
        const float lap = (dn[2] + dn[3]) - 2.0f * d;
        if (fabsf(lap) > p.depth_rel * d) e = 1;
      }
    }
    E[y * W + x] = e;
  }
}

}  // namespace

cudaError_t launch_edges(const EdgeParams& p, const float* depth, const void* normal, int half_normal,
                         const void* smap, int half_smap, uint8_t* E, cudaStream_t s) {
  dim3 block(TX, TY), grid((p.v.W + TX - 1) / TX, (p.v.H + TY - 1) / TY);
  if (!p.ssm) {
    dim3 dgrid((p.v.W + TX - 1) / TX, (p.v.H + TY * ER - 1) / (TY * ER));
    if (half_normal) edges_direct_kernel<half4><<<dgrid, block, 0, s>>>(p, depth, (const half4*)normal, E);
    else edges_direct_kernel<float4><<<dgrid, block, 0, s>>>(p, depth, (const float4*)normal, E);
  } else if (half_normal) {
    if (half_smap)
      edges_kernel<half4, __half><<<grid, block, 0, s>>>(p, depth, (const half4*)normal, (const __half*)smap, E);
    else
      edges_kernel<half4, float><<<grid, block, 0, s>>>(p, depth, (const half4*)normal, (const float*)smap, E);
  } else {
    if (half_smap)
      edges_kernel<float4, __half><<<grid, block, 0, s>>>(p, depth, (const float4*)normal, (const __half*)smap, E);
    else
      edges_kernel<float4, float><<<grid, block, 0, s>>>(p, depth, (const float4*)normal, (const float*)smap, E);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mrr
