// Tensor-core form of the dense prism / tetrahedron kernels (FP32 values).
//
// The operator contractions of the FR right-hand side (Section 2):
//   Eq. (disu)     u_f = M0 u
//   Eq. (FRfinal)  div = sum_d D_d f~_d + LIFT (F^C - n~ . M0 f~)
//   gradient path  grad~ u = D u + LIFT (n~ (u^C - u_f)), then M0 grad u
// run as tcgen05 kind::tf32 MMAs with the three-term split (A = Ah + Al,
// B = Bh + Bl, D = Al Bh + Ah Bl + Ah Bh, FP32 accumulation in TMEM).
//
// Roles: A is an operator (rows = output points, padded to an MMA height of
// 64 or 128; K = input points), staged once per persistent CTA in the
// canonical K-major layout without swizzle; B is the data of E elements
// (rows = (variable, element) columns, K = input points), written every tile
// by the CTA's threads in the 128-byte-swizzled K-major layout.  TMEM lane m
// of an accumulator is output point m, TMEM column n is data row n.
//
// Flux points enter K in a face-aligned order: the points of each face start
// on a multiple of 8, so that one 8-wide K slice never spans two faces and
// the lift of the gradient path can be taken face by face, each face's
// (constant) reference normal being applied in the epilogue.
#pragma once
#include <cstdint>
#include <type_traits>

#include "fr_hex.cuh"
#include "fr_kernels.cuh"
#include "fr_tc.cuh"

namespace frgb {

__host__ __device__ constexpr int tc_ru(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int tc_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int tc_pow2(int x) {
  int c = 32;
  while (c < x) c *= 2;
  return c;
}

// Face-aligned K extent of the flux points and face count of the prism and
// tetrahedron of order p = 1..8, identified by (nupts, nfpts); 0 otherwise.
__host__ __device__ constexpr int tc_kfp(int nu, int nf) {
  for (int p = 1; p <= 8; ++p) {
    const int nt = (p + 1) * (p + 2) / 2, nq = (p + 1) * (p + 1);
    if (nu == nq * (p + 2) / 2 && nf == 2 * nt + 3 * nq)
      return 2 * tc_ru(nt, 8) + 3 * tc_ru(nq, 8);
    if (nu == nt * (p + 3) / 3 && nf == 4 * nt) return 4 * tc_ru(nt, 8);
  }
  return 0;
}

__host__ __device__ constexpr int tc_nface(int nu, int nf) {
  for (int p = 1; p <= 8; ++p) {
    const int nt = (p + 1) * (p + 2) / 2, nq = (p + 1) * (p + 1);
    if (nu == nq * (p + 2) / 2 && nf == 2 * nt + 3 * nq) return 5;
    if (nu == nt * (p + 3) / 3 && nf == 4 * nt) return 4;
  }
  return 0;
}

// order p of the prism / tetrahedron with (nupts, nfpts); 0 otherwise
__host__ __device__ constexpr int tc_order(int nu, int nf) {
  for (int p = 1; p <= 8; ++p) {
    const int nt = (p + 1) * (p + 2) / 2, nq = (p + 1) * (p + 1);
    if (nu == nq * (p + 2) / 2 && nf == 2 * nt + 3 * nq) return p;
    if (nu == nt * (p + 3) / 3 && nf == 4 * nt) return p;
  }
  return 0;
}

// flux points on face fa: prisms list the two triangles, then the three
// quadrilaterals; tetrahedra four triangles
__host__ __device__ constexpr int tc_face_n(int nu, int nf, int fa) {
  const int p = tc_order(nu, nf);
  const int nt = (p + 1) * (p + 2) / 2, nq = (p + 1) * (p + 1);
  return tc_nface(nu, nf) == 5 ? (fa < 2 ? nt : nq) : nt;
}

// face-aligned K position of flux point f, and its inverse (-1: padding)
__host__ __device__ constexpr int tc_fpad(int nu, int nf, int f) {
  int fa = 0, f0 = 0, k0 = 0;
  while (f >= f0 + tc_face_n(nu, nf, fa)) {
    f0 += tc_face_n(nu, nf, fa);
    k0 += tc_ru(tc_face_n(nu, nf, fa), 8);
    ++fa;
  }
  return k0 + (f - f0);
}

__host__ __device__ constexpr int tc_kinv(int nu, int nf, int k) {
  int f0 = 0, k0 = 0;
  for (int fa = 0; fa < tc_nface(nu, nf); ++fa) {
    const int n = tc_face_n(nu, nf, fa);
    if (k < k0 + tc_ru(n, 8)) return k - k0 < n ? f0 + (k - k0) : -1;
    f0 += n;
    k0 += tc_ru(n, 8);
  }
  return -1;
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E, typename F>
__device__ __forceinline__ void tc_static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    tc_static_for<B + 1, E>(f);
  }
}

// Operator image: [M0 hi | M0 lo | D3 hi | D3 lo | L hi | L lo] (floats)
//   M0  MF x KU    M0[f][q]
//   D3  MU x 3KU   D_d[z][q] at column d KU + q
//   L   MU x KFP   LIFT[z][f] at column fpad[f]
template <int NU, int NF>
struct TcShape {
  static constexpr int KU = tc_ru(NU, 8), K3 = 3 * KU;
  static constexpr int KFP = tc_kfp(NU, NF), NFACE = tc_nface(NU, NF);
  static constexpr int MU = NU <= 64 ? 64 : 128, MF = NF <= 64 ? 64 : 128;
  static constexpr int SZ_M0 = MF * KU, SZ_D3 = MU * K3, SZ_L = MU * KFP;
  static constexpr int OPS = 2 * (SZ_M0 + SZ_D3 + SZ_L);
  static constexpr bool kShapeOk =
      KFP > 0 && NU >= 10 && NU <= 128 && NF <= 128 && KFP <= 128;
};

// Per-type flux-point ordering and face normals (kernel parameter).
struct TcGeom {
  uint8_t fpad[128];   // face-aligned K position of flux point f
  uint8_t pad[128];    // K positions in [0, KFP) holding no flux point
  int npad;
  int fslice[7];       // K slices (of 8) of face i: [fslice[i], fslice[i+1])
  float nface[6][3];   // reference outward normal of face i
};

constexpr size_t kTcSmemMax = 232448;  // dynamic shared memory per CTA
constexpr size_t kTcSmemSm = 233472;   // shared memory per SM

// Volume kernel: E elements per tile, B rows k E + el.
template <int NU, int NF, int E>
struct TcVolCfg {
  using S = TcShape<NU, NF>;
  static constexpr int NC = 5 * E, NCP = tc_ru(NC, 16);
  static constexpr int KB = tc_ru(tc_max(tc_max(S::K3, S::KFP), S::KU), 32);
  static constexpr int BFL = NCP * KB;  // floats per plane (hi or lo)
  static constexpr size_t SMEM = (size_t(S::OPS) + 2 * size_t(BFL)) * 4 + 1024;
  static constexpr int TCOLS = tc_pow2(4 * NCP);
  static constexpr bool kOk = S::kShapeOk && SMEM <= kTcSmemMax && E % 4 == 0 &&
                              NCP <= 256 && 4 * NCP <= 512;
};

// Gradient kernel: phase 1 B = [U (NCP x KBU) | DU (NCP x KBF)], phase 2
// B2 = physical gradient (N2 rows (j,k) E + el, K = KU) over the same planes.
template <int NU, int NF, int E>
struct TcGradCfg {
  using S = TcShape<NU, NF>;
  static constexpr int NC = 5 * E, NCP = tc_ru(NC, 16), N2 = tc_ru(15 * E, 16);
  static constexpr int KBU = tc_ru(S::KU, 32), KBF = tc_ru(S::KFP, 32);
  static constexpr int BFL = tc_max(NCP * (KBU + KBF), N2 * KBU);
  static constexpr size_t SMEM = (size_t(S::OPS) + 2 * size_t(BFL)) * 4 + 1024;
  static constexpr int TCOLS = tc_pow2(tc_max((3 + S::NFACE) * NCP, N2));
  static constexpr bool kOk = S::kShapeOk && SMEM <= kTcSmemMax && E % 4 == 0 &&
                              N2 <= 256 && (3 + S::NFACE) * NCP <= 512;
};

// Elements per tile: the largest of 16 / 12 / 8 / 4 whose shared memory
// and TMEM columns fit one CTA per SM.  Larger tiles put more elements in
// flight per SM and amortise each tile's chain of dependent phases; with
// four-element tiles (two CTAs per SM) the tetrahedron kernels ran 2.4x
// slower than with these.
template <int NU, int NF>
constexpr int tc_vol_epb() {
  return TcVolCfg<NU, NF, 16>::kOk   ? 16
         : TcVolCfg<NU, NF, 12>::kOk ? 12
         : TcVolCfg<NU, NF, 8>::kOk  ? 8
         : TcVolCfg<NU, NF, 4>::kOk  ? 4
                                     : 0;
}

template <int NU, int NF>
constexpr int tc_grad_epb() {
  return TcGradCfg<NU, NF, 16>::kOk   ? 16
         : TcGradCfg<NU, NF, 12>::kOk ? 12
         : TcGradCfg<NU, NF, 8>::kOk  ? 8
         : TcGradCfg<NU, NF, 4>::kOk  ? 4
                                      : 0;
}

// resident CTAs per SM: two when both shared memory and the 512 TMEM
// columns allow it
template <int NU, int NF, int E>
constexpr int tc_minb_vol() {
  return 2 * (TcVolCfg<NU, NF, E>::SMEM + 1024) <= kTcSmemSm &&
                 2 * TcVolCfg<NU, NF, E>::TCOLS <= 512
             ? 2
             : 1;
}

template <int NU, int NF, int E>
constexpr int tc_minb_grad() {
  return 2 * (TcGradCfg<NU, NF, E>::SMEM + 1024) <= kTcSmemSm &&
                 2 * TcGradCfg<NU, NF, E>::TCOLS <= 512
             ? 2
             : 1;
}

constexpr int kTcThreads = 256;

__device__ __forceinline__ float* tc_align1024(unsigned char* raw) {
  const uint32_t a = smem_u32(raw);
  return reinterpret_cast<float*>(raw + ((1024u - (a & 1023u)) & 1023u));
}

// TMEM row of this thread for an accumulator of height M (64 or 128): lane l
// of warp w holds row 32 (w mod 4) + l (M = 128) or 16 (w mod 4) + l for
// l < 16 (M = 64); -1 when the lane holds no row.
template <int M>
__device__ __forceinline__ int tc_row(int warp, int lane) {
  return M == 128 ? 32 * (warp & 3) + lane : (lane < 16 ? 16 * (warp & 3) + lane : -1);
}

// addresses of the 4-column chunks (k E + 4g .. +3) for k = 0..4 of the
// accumulator starting at column `col`
template <int E>
__device__ __forceinline__ void tc_chunk_addrs(uint32_t base, int col, int g,
                                               uint32_t a[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) a[k] = base + uint32_t(col + k * E + 4 * g);
}

// Stage the operator image and clear the B planes; set up the mbarrier and
// TMEM.  Returns the TMEM base address.
template <int OPS, int BFL2, int TCOLS>
__device__ __forceinline__ uint32_t tc_prologue(const float* __restrict__ opimg,
                                                float* ops, float* b,
                                                uint64_t* mbar, uint32_t* tslot) {
  const int tid = threadIdx.x;
  const float4* src = reinterpret_cast<const float4*>(opimg);
  float4* dst = reinterpret_cast<float4*>(ops);
  for (int i = tid; i < OPS / 4; i += blockDim.x) dst[i] = src[i];
  float4* bz = reinterpret_cast<float4*>(b);
  for (int i = tid; i < BFL2 / 4; i += blockDim.x) bz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  if ((tid >> 5) == 0) tmem_alloc(tslot, TCOLS);
  tc_sync_for_mma();
  return *tslot;
}

template <int TCOLS>
__device__ __forceinline__ void tc_epilogue(uint32_t tm, uint64_t* mbar,
                                            bool ok, int* flag) {
  if (!ok && threadIdx.x == 0) atomicOr(flag, 2);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tm, TCOLS);
  if (threadIdx.x == 0) mbar_inval(mbar);
}

// Transformed flux f~_d = S_d . F (Euler, plus the viscous part for NS) at
// one solution point from preloaded state, gradient and metric.
template <bool NS>
__device__ __forceinline__ void tc_point_flux(const float uz[5], const float g[3][5],
                                              const float Sm[9], const Phys<float>& ph,
                                              float ft[3][5]) {
  float F[3][5];
  euler_flux(uz, ph, F);
  if (NS) viscous_flux_acc(uz, g, ph, -1.f, F);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int k = 0; k < 5; ++k)
      ft[d][k] = Sm[3 * d] * F[0][k] + Sm[3 * d + 1] * F[1][k] + Sm[3 * d + 2] * F[2][k];
}

// ---------------------------------------------------------------------------
// Volume kernel: f~ = S F at the solution points, divergence with the
// correction lift, R = -div / J, the RK epilogue and the next stage's u_f.
// uin: stage input (FP32) or nullptr to read the register X (type TR).
template <int NU, int NF, int E, bool NS, typename TR, int MINB>
__global__ void __launch_bounds__(kTcThreads, MINB)
    k_vol_tc(long long ne, const float* __restrict__ uin,
             const float* __restrict__ grad, const float* __restrict__ fc,
             const float* __restrict__ smat, const float* __restrict__ rcpdjac,
             const float* __restrict__ opimg, const float* __restrict__ nref,
             TcGeom geo, Phys<float> ph, HexStage<float, TR> sa) {
  using S = TcShape<NU, NF>;
  using C = TcVolCfg<NU, NF, E>;
  constexpr int KU = S::KU, K3 = S::K3, KFP = S::KFP, NCP = C::NCP;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  float* m0h = tc_align1024(tc_raw);
  float* m0l = m0h + S::SZ_M0;
  float* d3h = m0l + S::SZ_M0;
  float* d3l = d3h + S::SZ_D3;
  float* lfh = d3l + S::SZ_D3;
  float* lfl = lfh + S::SZ_L;
  float* bh = lfl + S::SZ_L;
  float* bl = bh + C::BFL;
  const uint32_t tm = tc_prologue<S::OPS, 2 * C::BFL, C::TCOLS>(opimg, m0h, bh, &mbar, &tslot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, half = warp >> 2;
  const uint32_t tl = tm + (uint32_t(32 * (warp & 3)) << 16);
  constexpr uint32_t id_f = tc_idesc_tf32(S::MF, NCP), id_u = tc_idesc_tf32(S::MU, NCP);
  const int rf = tc_row<S::MF>(warp, lane), ru = tc_row<S::MU>(warp, lane);
  const bool fact = rf >= 0 && rf < NF;
  float nr[3] = {0.f, 0.f, 0.f};
  int fk = 0;
  if (fact) {
#pragma unroll
    for (int d = 0; d < 3; ++d) nr[d] = nref[rf * 3 + d];
    fk = geo.fpad[rf];
  }
  const TR* X = sa.X;
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (ne + E - 1) / E;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long e0 = tile * E;
    // (1) transformed flux -> B rows k E + el, K = d KU + z; PP points per
    //     thread and pass, all their loads issued before the flux arithmetic
    constexpr int PP = E * KU > kTcThreads ? 2 : 1;
    for (int i0 = tid; i0 < E * KU; i0 += PP * kTcThreads) {
      float uz[PP][5], g[PP][3][5], Sm[PP][9];
      bool live[PP];
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const int i = i0 + p * kTcThreads;
        const int el = i / KU, z = i - el * KU;
        const long long e = e0 + el;
        live[p] = i < E * KU && z < NU && e < ne;
        if (live[p]) {
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const long long ix = (e * 5 + k) * NU + z;
            uz[p][k] = uin ? uin[ix] : float(X[ix]);
          }
          if (NS) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int k = 0; k < 5; ++k) g[p][j][k] = grad[(e * 15 + j * 5 + k) * NU + z];
          }
#pragma unroll
          for (int r = 0; r < 9; ++r) Sm[p][r] = smat[(e * 9 + r) * NU + z];
        }
      }
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const int i = i0 + p * kTcThreads;
        if (i >= E * KU) continue;
        const int el = i / KU, z = i - el * KU;
        float ft[3][5];
        if (live[p]) {
          tc_point_flux<NS>(uz[p], g[p], Sm[p], ph, ft);
        } else {
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) ft[d][k] = 0.f;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int k = 0; k < 5; ++k) put_split(bh, bl, NCP, k * E + el, d * KU + z, ft[d][k]);
      }
    }
    tc_sync_for_mma();
    if (tid == 0) {
      // G_d = M0 f~_d at the flux points (columns d NCP), div = D3 f~ (3 NCP)
#pragma unroll 1
      for (int d = 0; d < 3; ++d)
#pragma unroll 1
        for (int s = 0; s < KU / 8; ++s)
          mma3(tm + d * NCP, m0h, m0l, KU, s, bh, bl, NCP, d * (KU / 8) + s, id_f, s > 0);
#pragma unroll 1
      for (int s = 0; s < K3 / 8; ++s)
        mma3(tm + 3 * NCP, d3h, d3l, K3, s, bh, bl, NCP, s, id_u, s > 0);
      tc_commit(&mbar);
    }
    ok = tc_wait_all(&mbar, phase);
    phase ^= 1;
    if (!ok) break;
    // (2) jm = F^C - n~ . G at the flux points -> B rows k E + el, K = fpad[f]
    for (int g = half; g < E / 4; g += 2) {
      float fcv[4][5];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long e = e0 + 4 * g + j;
#pragma unroll
        for (int k = 0; k < 5; ++k)
          fcv[j][k] = (fact && e < ne) ? fc[(e * 5 + k) * NF + rf] : 0.f;
      }
      float G[3][5][4];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        uint32_t a[5];
        tc_chunk_addrs<E>(tl, d * NCP, g, a);
        tmem_ld4x5(a, G[d]);
      }
      if (fact) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int el = 4 * g + j;
          const bool live = e0 + el < ne;
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const float v =
                live ? fcv[j][k] - (nr[0] * G[0][k][j] + nr[1] * G[1][k][j] +
                                    nr[2] * G[2][k][j])
                     : 0.f;
            put_split(bh, bl, NCP, k * E + el, fk, v);
          }
        }
      }
    }
    for (int i = tid; i < NCP * geo.npad; i += blockDim.x) {
      const int r = i / geo.npad;
      put_split(bh, bl, NCP, r, geo.pad[i - r * geo.npad], 0.f);
    }
    tc_sync_for_mma();
    if (tid == 0) {
#pragma unroll 1
      for (int s = 0; s < KFP / 8; ++s)
        mma3(tm + 3 * NCP, lfh, lfl, KFP, s, bh, bl, NCP, s, id_u, true);
      tc_commit(&mbar);
    }
    ok = tc_wait_all(&mbar, phase);
    phase ^= 1;
    if (!ok) break;
    // (3) R = -div / J, RK update; next stage value -> B rows k E + el, K = z
    const bool next = sa.uf_next != nullptr;
    for (int g = half; g < E / 4; g += 2) {
      float rj[4];
      TR xr[4][5], ar[4][5];
      bool live[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long e = e0 + 4 * g + j;
        live[j] = ru >= 0 && ru < NU && e < ne;
        rj[j] = live[j] ? rcpdjac[e * NU + ru] : 0.f;
        if (live[j]) {
          hex_stage_load(sa, e * 5 * NU + ru, NU, xr[j], ar[j]);
        } else {
#pragma unroll
          for (int k = 0; k < 5; ++k) xr[j][k] = ar[j][k] = TR(0);
        }
      }
      float dv[5][4];
      uint32_t a[5];
      tc_chunk_addrs<E>(tl, 3 * NCP, g, a);
      tmem_ld4x5(a, dv);
      if (ru >= 0 && ru < KU) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int el = 4 * g + j;
          const long long e = e0 + el;
          float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
          if (live[j]) {
            float R[5];
            const float u0[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 5; ++k) R[k] = -dv[k][j] * rj[j];
            hex_stage_apply(sa, e * 5 * NU + ru, NU, u0, R, xr[j], ar[j], s);
          }
          if (next) {
#pragma unroll
            for (int k = 0; k < 5; ++k) put_split(bh, bl, NCP, k * E + el, ru, s[k]);
          }
        }
      }
    }
    if (next) {
      tc_sync_for_mma();
      if (tid == 0) {
#pragma unroll 1
        for (int s = 0; s < KU / 8; ++s)
          mma3(tm, m0h, m0l, KU, s, bh, bl, NCP, s, id_f, s > 0);
        tc_commit(&mbar);
      }
      ok = tc_wait_all(&mbar, phase);
      phase ^= 1;
      if (!ok) break;
      // (4) u_f of the next stage
      for (int g = half; g < E / 4; g += 2) {
        float v[5][4];
        uint32_t a[5];
        tc_chunk_addrs<E>(tl, 0, g, a);
        tmem_ld4x5(a, v);
        if (fact) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const long long e = e0 + 4 * g + j;
            if (e < ne) {
#pragma unroll
              for (int k = 0; k < 5; ++k) sa.uf_next[(e * 5 + k) * NF + rf] = v[k][j];
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_epilogue<C::TCOLS>(tm, &mbar, ok, sa.flag);
}

// ---------------------------------------------------------------------------
// NS gradient kernel: corrected reference gradient D_d u + LIFT (n~_d du)
// (the lift taken per face with the face's constant normal), physical
// gradient (1/J) S^T grad~ u at the solution points, its values at the flux
// points M0 grad u, and the viscous normal flux q there.
template <int NU, int NF, int E, typename TR, int MINB>
__global__ void __launch_bounds__(kTcThreads, MINB)
    k_grad_tc(long long ne, const float* __restrict__ uin, const TR* __restrict__ X,
              const float* __restrict__ du, const float* __restrict__ smat,
              const float* __restrict__ rcpdjac, const float* __restrict__ opimg,
              TcGeom geo, float* __restrict__ grad, ViscArgs<float> va,
              BCTab<float> bc, Phys<float> ph, int* flag) {
  using S = TcShape<NU, NF>;
  using C = TcGradCfg<NU, NF, E>;
  constexpr int KU = S::KU, K3 = S::K3, KFP = S::KFP, NCP = C::NCP, N2 = C::N2;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  float* m0h = tc_align1024(tc_raw);
  float* m0l = m0h + S::SZ_M0;
  float* d3h = m0l + S::SZ_M0;
  float* d3l = d3h + S::SZ_D3;
  float* lfh = d3l + S::SZ_D3;
  float* lfl = lfh + S::SZ_L;
  float* bh = lfl + S::SZ_L;
  float* bl = bh + C::BFL;
  float* duh = bh + NCP * C::KBU;
  float* dul = bl + NCP * C::KBU;
  const uint32_t tm = tc_prologue<S::OPS, 2 * C::BFL, C::TCOLS>(opimg, m0h, bh, &mbar, &tslot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, half = warp >> 2;
  const uint32_t tl = tm + (uint32_t(32 * (warp & 3)) << 16);
  constexpr uint32_t id_u = tc_idesc_tf32(S::MU, NCP), id_2 = tc_idesc_tf32(S::MF, N2);
  const int rf = tc_row<S::MF>(warp, lane), ru = tc_row<S::MU>(warp, lane);
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (ne + E - 1) / E;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long e0 = tile * E;
    // (1) U: rows k E + el, K = z;  DU: rows k E + el, K = fpad[f]
    {
      constexpr int PU = (E * KU + kTcThreads - 1) / kTcThreads;
      constexpr int PF = (E * NF + kTcThreads - 1) / kTcThreads;
      float vu[PU][5], vf[PF][5];
#pragma unroll
      for (int p = 0; p < PU; ++p) {
        const int i = tid + p * kTcThreads;
        const int el = i / KU, z = i - el * KU;
        const long long e = e0 + el;
        const bool live = i < E * KU && z < NU && e < ne;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const long long ix = (e * 5 + k) * NU + z;
          vu[p][k] = live ? (uin ? uin[ix] : float(X[ix])) : 0.f;
        }
      }
#pragma unroll
      for (int p = 0; p < PF; ++p) {
        const int i = tid + p * kTcThreads;
        const int el = i / NF, f = i - el * NF;
        const long long e = e0 + el;
        const bool live = i < E * NF && e < ne;
#pragma unroll
        for (int k = 0; k < 5; ++k) vf[p][k] = live ? du[(e * 5 + k) * NF + f] : 0.f;
      }
#pragma unroll
      for (int p = 0; p < PU; ++p) {
        const int i = tid + p * kTcThreads;
        if (i < E * KU) {
          const int el = i / KU, z = i - el * KU;
#pragma unroll
          for (int k = 0; k < 5; ++k) put_split(bh, bl, NCP, k * E + el, z, vu[p][k]);
        }
      }
#pragma unroll
      for (int p = 0; p < PF; ++p) {
        const int i = tid + p * kTcThreads;
        if (i < E * NF) {
          const int el = i / NF, f = i - el * NF;
          const int kf = geo.fpad[f];
#pragma unroll
          for (int k = 0; k < 5; ++k) put_split(duh, dul, NCP, k * E + el, kf, vf[p][k]);
        }
      }
    }
    for (int i = tid; i < NCP * geo.npad; i += blockDim.x) {
      const int r = i / geo.npad;
      put_split(duh, dul, NCP, r, geo.pad[i - r * geo.npad], 0.f);
    }
    tc_sync_for_mma();
    if (tid == 0) {
#pragma unroll 1
      for (int d = 0; d < 3; ++d)
#pragma unroll 1
        for (int s = 0; s < KU / 8; ++s)
          mma3(tm + d * NCP, d3h, d3l, K3, d * (KU / 8) + s, bh, bl, NCP, s, id_u, s > 0);
#pragma unroll 1
      for (int fa = 0; fa < S::NFACE; ++fa)
#pragma unroll 1
        for (int s = geo.fslice[fa]; s < geo.fslice[fa + 1]; ++s)
          mma3(tm + (3 + fa) * NCP, lfh, lfl, KFP, s, duh, dul, NCP, s, id_u,
               s > geo.fslice[fa]);
      tc_commit(&mbar);
    }
    ok = tc_wait_all(&mbar, phase);
    phase ^= 1;
    if (!ok) break;
    // (2) physical gradient at the solution points -> grad, B2 rows
    //     (j 5 + k) E + el, K = z
    for (int g = half; g < E / 4; g += 2) {
      float Sm[4][9], rj[4];
      bool live[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long e = e0 + 4 * g + j;
        live[j] = ru >= 0 && ru < NU && e < ne;
#pragma unroll
        for (int r = 0; r < 9; ++r) Sm[j][r] = live[j] ? smat[(e * 9 + r) * NU + ru] : 0.f;
        rj[j] = live[j] ? rcpdjac[e * NU + ru] : 0.f;
      }
      float gr[3][5][4];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        uint32_t a[5];
        tc_chunk_addrs<E>(tl, d * NCP, g, a);
        tmem_ld4x5(a, gr[d]);
      }
#pragma unroll 1
      for (int fa = 0; fa < S::NFACE; ++fa) {
        float t[5][4];
        uint32_t a[5];
        tc_chunk_addrs<E>(tl, (3 + fa) * NCP, g, a);
        tmem_ld4x5(a, t);
        const float n0 = geo.nface[fa][0], n1 = geo.nface[fa][1], n2 = geo.nface[fa][2];
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            gr[0][k][j] += n0 * t[k][j];
            gr[1][k][j] += n1 * t[k][j];
            gr[2][k][j] += n2 * t[k][j];
          }
      }
      if (ru >= 0 && ru < KU) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int el = 4 * g + j;
          const long long e = e0 + el;
          float gg[3][5];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 5; ++k) gg[c][k] = 0.f;
          if (live[j]) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int k = 0; k < 5; ++k) {
                gg[c][k] = rj[j] * (Sm[j][c] * gr[0][k][j] + Sm[j][3 + c] * gr[1][k][j] +
                                    Sm[j][6 + c] * gr[2][k][j]);
                grad[(e * 15 + c * 5 + k) * NU + ru] = gg[c][k];
              }
          }
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 5; ++k)
              put_split(bh, bl, N2, (c * 5 + k) * E + el, ru, gg[c][k]);
        }
      }
    }
    tc_sync_for_mma();
    if (tid == 0) {
#pragma unroll 1
      for (int s = 0; s < KU / 8; ++s)
        mma3(tm, m0h, m0l, KU, s, bh, bl, N2, s, id_2, s > 0);
      tc_commit(&mbar);
    }
    ok = tc_wait_all(&mbar, phase);
    phase ^= 1;
    if (!ok) break;
    // (3) gradient at the flux points -> viscous normal flux q
    for (int g = half; g < E / 4; g += 2) {
      float ut[4][5], nv[4][3];
      int fb[4];
      bool live[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long e = e0 + 4 * g + j;
        live[j] = rf >= 0 && rf < NF && e < ne;
#pragma unroll
        for (int k = 0; k < 5; ++k) ut[j][k] = live[j] ? va.uf[(e * 5 + k) * NF + rf] : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) nv[j][c] = live[j] ? va.fnv[(e * 3 + c) * NF + rf] : 0.f;
        fb[j] = live[j] ? va.fbc[e * NF + rf] : -1;
      }
      float gf[3][5][4];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        uint32_t a[5];
        tc_chunk_addrs<E>(tl, 5 * b * E, g, a);
        tmem_ld4x5(a, gf[b]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!live[j]) continue;
        const long long e = e0 + 4 * g + j;
        float G[3][5], q[5];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 5; ++k) G[c][k] = gf[c][k][j];
        visc_q_pre(bc, ph, ut[j], G, nv[j], fb[j], q, prescribed_at(va, e, rf, NF));
#pragma unroll
        for (int k = 0; k < 5; ++k) va.q[(e * 5 + k) * NF + rf] = q[k];
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_epilogue<C::TCOLS>(tm, &mbar, ok, flag);
}

// ---------------------------------------------------------------------------
// Volume kernel with the data as the MMA's A operand.  A = data of E
// elements, row el 5 + k (element el, variable k; M = 128 rows: E = 25,
// M = 64: E = 12), K = input points, 128-byte swizzle; B = operator, rows =
// output points padded to 16, canonical K-major layout.  TMEM lane r holds
// data row r and columns are output points, so every epilogue thread owns
// one (element, variable) row and reads and writes it with contiguous
// 16-byte accesses.  Operator image as TcShape but with row counts NUN /
// NFN (ru16).
template <int NU, int NF, int M>
struct TcaVolCfg {
  using S = TcShape<NU, NF>;
  static constexpr int E = M / 5, ROWS = 5 * E;
  static constexpr int NUN = tc_ru(NU, 16), NFN = tc_ru(NF, 16);
  static constexpr int SZ_M0 = NFN * S::KU, SZ_D3 = NUN * S::K3, SZ_L = NUN * S::KFP;
  static constexpr int OPS = 2 * (SZ_M0 + SZ_D3 + SZ_L);
  static constexpr int KA = tc_ru(tc_max(tc_max(S::K3, S::KFP), S::KU), 32);
  static constexpr int AFL = M * KA;  // floats per A plane
  static constexpr size_t SMEM =
      (size_t(OPS) + 2 * size_t(AFL) + size_t(tc_ru(3 * NF, 4))) * 4 + 1024;
  static constexpr int TCOLS = tc_pow2(3 * NFN + NUN);
  static constexpr bool kOk = S::kShapeOk && SMEM <= kTcSmemMax && 3 * NFN + NUN <= 512 &&
                              NFN <= 256 && NUN <= 256 && S::KU % 4 == 0;
};

template <int NU, int NF>
constexpr int tca_m() {
  return TcaVolCfg<NU, NF, 128>::kOk ? 128 : TcaVolCfg<NU, NF, 64>::kOk ? 64 : 0;
}

// D (+)= A B^T, A = data (128-byte swizzle, R rows), B = operator
// (canonical, K columns), K slice sa of A and sb of B
__device__ __forceinline__ void mma3a(uint32_t d, const float* ah, const float* al,
                                      int R, int sa, const float* bh, const float* bl,
                                      int K, int sb, uint32_t idesc, bool acc) {
  const uint32_t sbo = uint32_t(K / 4) * 128u;
  const uint64_t a_h = tc_desc_sw128(ah, R, sa), a_l = tc_desc_sw128(al, R, sa);
  const uint64_t b_h = tc_desc(bh + sb * 64, 128, sbo);
  const uint64_t b_l = tc_desc(bl + sb * 64, 128, sbo);
  tc_mma_tf32(d, a_l, b_h, idesc, acc);
  tc_mma_tf32(d, a_h, b_l, idesc, true);
  tc_mma_tf32(d, a_h, b_h, idesc, true);
}

// four consecutive K values (k0 a multiple of 4) of row r as TF32 pairs
__device__ __forceinline__ void put_split4(float* hi, float* lo, int R, int r, int k0,
                                           float4 x) {
  const int o = sw128_offset(r, k0, R);
  float4 h, l;
  h.x = tf32_hi(x.x); l.x = tf32_hi(x.x - h.x);
  h.y = tf32_hi(x.y); l.y = tf32_hi(x.y - h.y);
  h.z = tf32_hi(x.z); l.z = tf32_hi(x.z - h.z);
  h.w = tf32_hi(x.w); l.w = tf32_hi(x.w - h.w);
  *reinterpret_cast<float4*>(hi + o) = h;
  *reinterpret_cast<float4*>(lo + o) = l;
}

// n consecutive values of a row from global memory: 16-byte loads when n
// and the address allow it
template <int N>
__device__ __forceinline__ void tc_row_load(const float* __restrict__ src, bool vec,
                                            float v[N]) {
  if (N % 4 == 0 && vec) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 q = reinterpret_cast<const float4*>(src)[i];
      v[4 * i] = q.x;
      v[4 * i + 1] = q.y;
      v[4 * i + 2] = q.z;
      v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = src[i];
  }
}

template <int N>
__device__ __forceinline__ void tc_row_store(float* __restrict__ dst, bool vec,
                                             const float v[N]) {
  if (N % 4 == 0 && vec) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      reinterpret_cast<float4*>(dst)[i] =
          make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) dst[i] = v[i];
  }
}

// RK epilogue of one variable over the N points of an element row at i0
// (the arithmetic of hex_stage_apply, FP32 registers), from the register
// values x (X) and ac (A) read beforehand; s receives the next stage value.
template <int N>
__device__ __forceinline__ void tc_stage_row(const HexStage<float, float>& a,
                                             long long i0, bool vec, const float R[N],
                                             const float x[N], const float ac[N],
                                             float s[N]) {
  if (a.mode == 0) {
    tc_row_store<N>(a.out + i0, vec, R);
#pragma unroll
    for (int z = 0; z < N; ++z) s[z] = 0.f;
    return;
  }
  const float dt = float(*a.dt);
  const int st = a.stage;
  if (a.mode == 1) {
    if (st < 3) {
      float ao[N];
#pragma unroll
      for (int z = 0; z < N; ++z) {
        const float r = R[z];
        if (st == 0) {
          ao[z] = x[z] + dt * float(1.0 / 6.0) * r;
          s[z] = x[z] + dt * 0.5f * r;
        } else {
          ao[z] = ac[z] + dt * float(1.0 / 3.0) * r;
          s[z] = x[z] + (st == 1 ? dt * 0.5f : dt) * r;
        }
      }
      tc_row_store<N>(a.A + i0, vec, ao);
      tc_row_store<N>(a.Y + i0, vec, s);
    } else {
#pragma unroll
      for (int z = 0; z < N; ++z) s[z] = ac[z] + dt * float(1.0 / 6.0) * R[z];
      tc_row_store<N>(a.X + i0, vec, s);
    }
    return;
  }
  const float b = float(c_rk45_b[st]);
  const float am = st < 4 ? float(c_rk45_a[st]) - b : 0.f;
  float xo[N];
#pragma unroll
  for (int z = 0; z < N; ++z) {
    xo[z] = x[z] + b * dt * R[z];
    s[z] = st < 4 ? xo[z] + am * dt * R[z] : xo[z];
  }
  tc_row_store<N>(a.X + i0, vec, xo);
  if (st < 4) tc_row_store<N>(a.Y + i0, vec, s);
  if (a.E) {  // error estimate dt sum_i (b_i - bhat_i) R_i
    const float ec = float(c_rk45_e[st]);
    float ev[N];
    if (st > 0) {
      tc_row_load<N>(a.E + i0, vec, ev);
    } else {
#pragma unroll
      for (int z = 0; z < N; ++z) ev[z] = 0.f;
    }
#pragma unroll
    for (int z = 0; z < N; ++z) ev[z] = st == 0 ? ec * dt * R[z] : ev[z] + ec * dt * R[z];
    tc_row_store<N>(a.E + i0, vec, ev);
  }
}

template <int NU, int NF, int M, bool NS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_vol_tca(long long ne, const float* __restrict__ uin,
              const float* __restrict__ grad, const float* __restrict__ fc,
              const float* __restrict__ smat, const float* __restrict__ rcpdjac,
              const float* __restrict__ opimg, const float* __restrict__ nref,
              Phys<float> ph, HexStage<float, float> sa) {
  using S = TcShape<NU, NF>;
  using C = TcaVolCfg<NU, NF, M>;
  constexpr int E = C::E, KU = S::KU, K3 = S::K3, KFP = S::KFP;
  constexpr int NUN = C::NUN, NFN = C::NFN;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  float* m0h = tc_align1024(tc_raw);
  float* m0l = m0h + C::SZ_M0;
  float* d3h = m0l + C::SZ_M0;
  float* d3l = d3h + C::SZ_D3;
  float* lfh = d3l + C::SZ_D3;
  float* lfl = lfh + C::SZ_L;
  float* ah = lfl + C::SZ_L;  // 1024-aligned: OPS is a multiple of 256
  float* al = ah + C::AFL;
  float* nrs = al + C::AFL;   // [NF][3] reference normals
  const uint32_t tm = tc_prologue<C::OPS, 2 * C::AFL, C::TCOLS>(opimg, m0h, ah, &mbar, &tslot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 3 * NF; i += blockDim.x) nrs[i] = nref[i];
  __syncthreads();
  const uint32_t tl = tm + (uint32_t(32 * (warp & 3)) << 16);
  constexpr uint32_t id_f = tc_idesc_tf32(M, NFN), id_u = tc_idesc_tf32(M, NUN);
  const bool epi = warp < 4;  // warps 0-3 (one per TMEM lane quarter) run the epilogues
  const int row = tc_row<M>(warp, lane);  // data row of this thread's TMEM lane
  const int rel = row >= 0 ? row / 5 : 0, rk = row >= 0 ? row - 5 * rel : 0;
  const bool vf = (reinterpret_cast<unsigned long long>(fc) & 15u) == 0;
  const bool vu = (reinterpret_cast<unsigned long long>(sa.X) & 15u) == 0 &&
                  (reinterpret_cast<unsigned long long>(sa.Y) & 15u) == 0 &&
                  (reinterpret_cast<unsigned long long>(sa.A) & 15u) == 0 &&
                  (reinterpret_cast<unsigned long long>(sa.out) & 15u) == 0 &&
                  (reinterpret_cast<unsigned long long>(rcpdjac) & 15u) == 0;
  const bool vn = sa.uf_next == nullptr ||
                  (reinterpret_cast<unsigned long long>(sa.uf_next) & 15u) == 0;
  const float* X = sa.X;
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (ne + E - 1) / E;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long e0 = tile * E;
    const long long e = e0 + rel;
    const bool live = row >= 0 && row < C::ROWS && e < ne;
    // (1) transformed flux -> A rows el 5 + k, K = d KU + z
    constexpr int PP = E * KU > kTcThreads ? 2 : 1;
    for (int i0 = tid; i0 < E * KU; i0 += PP * kTcThreads) {
      float uz[PP][5], g[PP][3][5], Sm[PP][9];
      bool pl[PP];
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const int i = i0 + p * kTcThreads;
        const int el = i / KU, z = i - el * KU;
        const long long ee = e0 + el;
        pl[p] = i < E * KU && z < NU && ee < ne;
        if (pl[p]) {
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const long long ix = (ee * 5 + k) * NU + z;
            uz[p][k] = uin ? uin[ix] : X[ix];
          }
          if (NS) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int k = 0; k < 5; ++k) g[p][j][k] = grad[(ee * 15 + j * 5 + k) * NU + z];
          }
#pragma unroll
          for (int r = 0; r < 9; ++r) Sm[p][r] = smat[(ee * 9 + r) * NU + z];
        }
      }
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const int i = i0 + p * kTcThreads;
        if (i >= E * KU) continue;
        const int el = i / KU, z = i - el * KU;
        float ft[3][5];
        if (pl[p]) {
          tc_point_flux<NS>(uz[p], g[p], Sm[p], ph, ft);
        } else {
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int k = 0; k < 5; ++k) ft[d][k] = 0.f;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int k = 0; k < 5; ++k) put_split(ah, al, M, el * 5 + k, d * KU + z, ft[d][k]);
      }
    }
    tc_sync_for_mma();
    if (tid == 0) {
#pragma unroll 1
      for (int d = 0; d < 3; ++d)
#pragma unroll 1
        for (int s2 = 0; s2 < KU / 8; ++s2)
          mma3a(tm + d * NFN, ah, al, M, d * (KU / 8) + s2, m0h, m0l, KU, s2, id_f, s2 > 0);
#pragma unroll 1
      for (int s2 = 0; s2 < K3 / 8; ++s2)
        mma3a(tm + 3 * NFN, ah, al, M, s2, d3h, d3l, K3, s2, id_u, s2 > 0);
      tc_commit(&mbar);
    }
    ok = tc_wait_all(&mbar, phase);
    phase ^= 1;
    if (!ok) break;
    // (2) jump F^C - n~ . M0 f~ of this row at all flux points -> A row, K =
    //     face-aligned flux-point order
    if (epi) {
      float jv[NF];
      if (live) {
        tc_row_load<NF>(fc + (e * 5 + rk) * NF, vf, jv);
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) jv[f] = 0.f;
      }
      tc_static_for<0, NFN / 16>([&](auto CI) {
        constexpr int c = decltype(CI)::value;
        float g0[16], g1[16], g2[16];
        tmem_ld16(tl + 0 * NFN + 16 * c, g0);
        tmem_ld16(tl + 1 * NFN + 16 * c, g1);
        tmem_ld16(tl + 2 * NFN + 16 * c, g2);
        tc_static_for<0, 16>([&](auto II) {
          constexpr int i = decltype(II)::value, f = 16 * c + i;
          if constexpr (f < NF)
            jv[f] -= nrs[3 * f] * g0[i] + nrs[3 * f + 1] * g1[i] + nrs[3 * f + 2] * g2[i];
        });
      });
      if (row >= 0) {
        if (!live) {
#pragma unroll
          for (int f = 0; f < NF; ++f) jv[f] = 0.f;
        }
        tc_static_for<0, KFP / 4>([&](auto KC) {
          constexpr int k0 = 4 * decltype(KC)::value;
          constexpr int f0 = tc_kinv(NU, NF, k0), f1 = tc_kinv(NU, NF, k0 + 1);
          constexpr int f2 = tc_kinv(NU, NF, k0 + 2), f3 = tc_kinv(NU, NF, k0 + 3);
          float4 w;
          w.x = f0 >= 0 ? jv[f0 < 0 ? 0 : f0] : 0.f;
          w.y = f1 >= 0 ? jv[f1 < 0 ? 0 : f1] : 0.f;
          w.z = f2 >= 0 ? jv[f2 < 0 ? 0 : f2] : 0.f;
          w.w = f3 >= 0 ? jv[f3 < 0 ? 0 : f3] : 0.f;
          put_split4(ah, al, M, row, k0, w);
        });
      }
    }
    tc_sync_for_mma();
    if (tid == 0) {
#pragma unroll 1
      for (int s2 = 0; s2 < KFP / 8; ++s2)
        mma3a(tm + 3 * NFN, ah, al, M, s2, lfh, lfl, KFP, s2, id_u, true);
      tc_commit(&mbar);
    }
    ok = tc_wait_all(&mbar, phase);
    phase ^= 1;
    if (!ok) break;
    // (3) R = -div / J and the RK update of this row, 16 points at a time;
    //     next stage value -> A (K = z, zero beyond NU)
    const bool next = sa.uf_next != nullptr;
    if (epi) {
      bool nx, na;
      hex_stage_needs(sa, &nx, &na);
      const long long i0 = (e * 5 + rk) * NU;
      bool bad = false;
      tc_static_for<0, KU / 16 + (KU % 16 ? 1 : 0)>([&](auto CI) {
        constexpr int c = decltype(CI)::value, z0 = 16 * c;
        constexpr int n = NU - z0 < 16 ? (NU - z0 > 0 ? NU - z0 : 0) : 16;
        float sv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) sv[i] = 0.f;
        float t[16];
        if constexpr (z0 < NUN) tmem_ld16(tl + 3 * NFN + z0, t);
        if constexpr (n > 0) {
          if (live) {
            const bool vc = vu && NU % 4 == 0 && n % 4 == 0;
            float rj[n], R[n], xr[n], ar[n], so[n];
            tc_row_load<n>(rcpdjac + e * NU + z0, vc, rj);
            if (nx) {
              tc_row_load<n>(sa.X + i0 + z0, vc, xr);
            } else {
#pragma unroll
              for (int i = 0; i < n; ++i) xr[i] = 0.f;
            }
            if (na) {
              tc_row_load<n>(sa.A + i0 + z0, vc, ar);
            } else {
#pragma unroll
              for (int i = 0; i < n; ++i) ar[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < n; ++i) {
              R[i] = -t[i] * rj[i];
              bad |= !isfinite(R[i]);
            }
            tc_stage_row<n>(sa, i0 + z0, vc, R, xr, ar, so);
#pragma unroll
            for (int i = 0; i < n; ++i) sv[i] = so[i];
          }
        }
        if (next && row >= 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (z0 + 4 * q < KU)
              put_split4(ah, al, M, row, z0 + 4 * q,
                         make_float4(sv[4 * q], sv[4 * q + 1], sv[4 * q + 2], sv[4 * q + 3]));
        }
      });
      if (bad) atomicOr(sa.flag, 1);
    }
    if (next) {
      tc_sync_for_mma();
      if (tid == 0) {
#pragma unroll 1
        for (int s2 = 0; s2 < KU / 8; ++s2)
          mma3a(tm, ah, al, M, s2, m0h, m0l, KU, s2, id_f, s2 > 0);
        tc_commit(&mbar);
      }
      ok = tc_wait_all(&mbar, phase);
      phase ^= 1;
      if (!ok) break;
      // (4) u_f of the next stage, row by row, 16 flux points at a time
      if (epi) {
        tc_static_for<0, NFN / 16>([&](auto CI) {
          constexpr int f0 = 16 * decltype(CI)::value;
          constexpr int n = NF - f0 < 16 ? NF - f0 : 16;
          float t[16];
          tmem_ld16(tl + f0, t);
          if (live)
            tc_row_store<n>(sa.uf_next + (e * 5 + rk) * NF + f0, vn && NF % 4 == 0 && n % 4 == 0, t);
        });
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_epilogue<C::TCOLS>(tm, &mbar, ok, sa.flag);
}

}  // namespace frgb
