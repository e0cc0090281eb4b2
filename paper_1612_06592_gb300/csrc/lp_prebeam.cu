// Preliminary beams of station groups: the first stage of two-stage
// beamforming (Sec. 4, network paragraph).  Only a few 16-bit station streams
// fit through the link to the processing cluster, so disjoint groups of
// stations are first combined, each into one preliminary beam toward its own
// direction s_g, phased to the group's phase centre r_g (the mean position of
// its stations); the preliminary beams travel as complex int16 like station
// data and the final beams are formed from them by the ordinary pipeline with
// the group centres as station positions.
//
//     pb[p][k][m][g] = sum_{s in g} w1[k][s] x[p][k][m][s],
//     w1[k][s] = exp(-2 pi i nu_k ((r_s - r_g) . s_g) / c),
//     y = round half to even (scale * pb), saturated to [-32767, 32767].
//
// k_prebeam: one 4-warp block per (pol, subband, 256 frames), two frames per
// thread.  The tile's samples are read once from HBM (contiguous [frame][S],
// 16-byte chunks with several loads in flight per thread) into shared memory
// station-major, so that a thread reads both of its frames of one station in
// one access; the group sums run over the stations of each group in turn
// (member list sorted by group, weight and tile offset in one broadcast
// 16-byte load) with FP32 FMAs; the int16 codes
// are gathered in shared memory and written back as one contiguous
// [frame][group] range of the output.  HBM-bound: 2 S (int8) or 4 S (int16)
// bytes in and 4 G bytes out per frame, 8 S FLOP.
//
// k_prebeam_pairs (int8 input, S a multiple of 8, G = 4, 8 or 16, 16-byte
// aligned input and output): the same sums with about a third of the
// instructions per sample.  A thread owns a frame pair: it reads the pair's
// 16-byte chunks straight from HBM (through L1) and stores, per member
// station, one word holding both frames' (re, im) bytes into a member-major
// shared tile; the group sums then take one word, four byte-permutes, two
// paired FP32 adds and four paired FMAs per station for both frames; the codes
// are rounded by the 1.5 * 2^23 addition (round half to even, exact below
// 2^22) and leave the thread as 16-byte stores of its 2 G contiguous words.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "lp_internal.cuh"

struct lp_prebeam {
  int S = 0, P = 0, K = 0, G = 0, first_bin = 0, input_dtype = 0;
  long long F = 0;
  int device = -1;
  int E = 0;                            // stations in some group
  void* mem = nullptr;                  // the caller's workspace, carved below
  float2* w1 = nullptr;                 // [K][E] weights in member order
  int* member = nullptr;                // [E] station of member e (sorted by group)
  int* goff = nullptr;                  // [G + 1] first member of each group
  double* rel = nullptr;                // [E][3] r_s - r_g
  double* mdir = nullptr;               // [E][3] direction of the member's group
  unsigned long long* n_sat = nullptr;  // saturated int16 codes since the last read
  std::vector<double> centres;          // [G][3]
  bool groups_set = false;
  cudaStream_t last_stream = nullptr;
  std::string err;
};

namespace lp {
namespace {

constexpr int PB_NTH = 128;          // threads per block, two frames each
constexpr int PB_FT = 2 * PB_NTH;    // frames per block
constexpr int PB_FTP = PB_FT + 2;    // padded station row of the sample tile
constexpr int PB_YP = PB_FT + 1;     // padded group row of the output tile

template <typename T2> struct PbPair;
template <> struct PbPair<char2> { using T = char4; };
template <> struct PbPair<short2> { using T = short4; };

// int16 transport code of scale * v: round half to even, saturate to +-32767
// (|scale v| >= 32767.5 is exactly when the rounded value leaves the range)
__device__ __forceinline__ short pb_code(float v, float scale, int& sat) {
  const float s = v * scale;
  sat += fabsf(s) >= 32767.5f ? 1 : 0;
  return (short)__float2int_rn(fminf(fmaxf(s, -32767.f), 32767.f));
}

// One tile element (a station sample of one frame) into the station-major tile.
template <typename T2>
__device__ __forceinline__ void put_sample(T2* xs, int e, int S, T2 v) {
  const int fr = e / S;
  xs[(e - fr * S) * PB_FTP + fr] = v;
}

// Exact int8 / int16 -> FP32 without a conversion instruction: the sample plus
// its bias (2^7 or 2^15) is placed in the low mantissa bits of 2^23, and 2^23
// plus the bias is subtracted (all values involved are exact in FP32).
struct Pair4f {
  float a, b, c, d;   // elements 0..3 of a char4 / short4
};
__device__ __forceinline__ Pair4f to_f32(char4 q) {
  const uint32_t u = *reinterpret_cast<const uint32_t*>(&q) ^ 0x80808080u;
  constexpr float off = 8388608.0f + 128.0f;
  return {__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7650)) - off,
          __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7651)) - off,
          __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7652)) - off,
          __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7653)) - off};
}
__device__ __forceinline__ Pair4f to_f32(short4 q) {
  const uint2 u2 = *reinterpret_cast<const uint2*>(&q);
  const uint32_t lo = u2.x ^ 0x80008000u, hi = u2.y ^ 0x80008000u;
  constexpr float off = 8388608.0f + 32768.0f;
  return {__uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7610)) - off,
          __uint_as_float(__byte_perm(lo, 0x4B000000u, 0x7632)) - off,
          __uint_as_float(__byte_perm(hi, 0x4B000000u, 0x7610)) - off,
          __uint_as_float(__byte_perm(hi, 0x4B000000u, 0x7632)) - off};
}

template <typename T2>
__global__ void __launch_bounds__(PB_NTH) k_prebeam(
    const T2* __restrict__ x, const float2* __restrict__ w1, const int* __restrict__ member,
    const int* __restrict__ goff, int S, int K, int G, int E, long long F, float scale, int vec,
    short2* __restrict__ y, unsigned long long* __restrict__ n_sat) {
  using T4 = typename PbPair<T2>::T;
  constexpr int PER = 16 / sizeof(T2);                         // samples per 16-byte chunk
  extern __shared__ float4 pb_smem[];
  float4* ws = pb_smem;                                        // [E] (w.re, w.im, tile offset, 0)
  T2* xs = reinterpret_cast<T2*>(ws + E);                      // [S][PB_FTP]
  short2* ys = reinterpret_cast<short2*>(xs + (size_t)S * PB_FTP);   // [G][PB_YP]
  int* go = reinterpret_cast<int*>(ys + (size_t)G * PB_YP);   // [G + 1]

  const int tile = blockIdx.x, k = blockIdx.y, pol = blockIdx.z;
  const int tid = threadIdx.x;
  const long long f0 = (long long)tile * PB_FT;
  const int nvalid = (int)min((long long)PB_FT, F - f0);
  for (int e = tid; e < E; e += PB_NTH) {
    const float2 w = w1[(long long)k * E + e];
    ws[e] = make_float4(w.x, w.y, __int_as_float(member[e] * PB_FTP), 0.f);
  }
  for (int g = tid; g <= G; g += PB_NTH) go[g] = goff[g];
  // samples of this (pol, k) and frame tile -> xs[s][frame]: the tile is one
  // contiguous range of nvalid * S samples; with vec (16-byte aligned slabs)
  // it is read in 16-byte chunks, four loads in flight per thread before their
  // samples are stored, and the ragged end sample by sample
  const T2* xk = x + (((long long)pol * K + k) * F + f0) * S;
  const int n_el = nvalid * S;
  int done = 0;
  if (vec) {
    const int n_ch = n_el / PER;
    const uint4* xc = reinterpret_cast<const uint4*>(xk);
    // (frame, station) of the first sample of chunk c, kept for c = tid,
    // tid + PB_NTH, ... by adding PB_NTH * PER samples with a carry
    int fr_c = (tid * PER) / S, st_c = tid * PER - fr_c * S;
    const int dq = (PB_NTH * PER) / S, dr = PB_NTH * PER - dq * S;
    for (int c0 = tid; c0 < n_ch; c0 += 4 * PB_NTH) {
      uint4 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = c0 + i * PB_NTH;
        if (c < n_ch) v[i] = __ldg(xc + c);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = c0 + i * PB_NTH;
        if (c >= n_ch) break;
        const T2* el = reinterpret_cast<const T2*>(&v[i]);
        int fr = fr_c, st = st_c;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
          xs[st * PB_FTP + fr] = el[j];
          if (++st == S) {
            st = 0;
            ++fr;
          }
        }
        st_c += dr;
        fr_c += dq;
        if (st_c >= S) {
          st_c -= S;
          ++fr_c;
        }
      }
    }
    done = n_ch * PER;
  }
  for (int e = done + tid; e < n_el; e += PB_NTH) put_sample(xs, e, S, xk[e]);
  __syncthreads();

  const int fl = 2 * tid;                                      // my frames fl, fl + 1
  int sat = 0;
  for (int g = 0; g < G; ++g) {
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    const int e1 = go[g + 1];
#pragma unroll 2
    for (int e = go[g]; e < e1; ++e) {
      const float4 w = ws[e];                                  // broadcast
      const Pair4f q = to_f32(*reinterpret_cast<const T4*>(xs + __float_as_int(w.z) + fl));
      // (w.x + i w.y) (q.a + i q.b), frame fl;  (q.c + i q.d), frame fl + 1
      a0.x = fmaf(w.x, q.a, fmaf(-w.y, q.b, a0.x));
      a0.y = fmaf(w.x, q.b, fmaf(w.y, q.a, a0.y));
      a1.x = fmaf(w.x, q.c, fmaf(-w.y, q.d, a1.x));
      a1.y = fmaf(w.x, q.d, fmaf(w.y, q.c, a1.y));
    }
    // frames past the block end hold stale samples: their codes are never
    // written and their saturations not counted
    int s0 = 0, s1 = 0;
    short2 c0, c1;
    c0.x = pb_code(a0.x, scale, s0);
    c0.y = pb_code(a0.y, scale, s0);
    c1.x = pb_code(a1.x, scale, s1);
    c1.y = pb_code(a1.y, scale, s1);
    sat += (fl < nvalid ? s0 : 0) + (fl + 1 < nvalid ? s1 : 0);
    ys[g * PB_YP + fl] = c0;
    ys[g * PB_YP + fl + 1] = c1;
  }
  const int wsat = __reduce_add_sync(0xffffffffu, sat);
  if ((tid & 31) == 0 && wsat) atomicAdd(n_sat, (unsigned long long)wsat);
  __syncthreads();
  // [frame][group] codes of the valid frames: one contiguous output range
  short2* yk = y + (((long long)pol * K + k) * F + f0) * G;
  {
    int fr = tid / G, g = tid - fr * G;                        // (frame, group) of e
    const int dq = PB_NTH / G, dr = PB_NTH - dq * G;
    for (int e = tid; e < nvalid * G; e += PB_NTH) {
      yk[e] = ys[g * PB_YP + fr];
      g += dr;
      fr += dq;
      if (g >= G) {
        g -= G;
        ++fr;
      }
    }
  }
}

constexpr int PF_NTH = 128;          // threads per block = frame pairs per tile
constexpr int PF_FT = 2 * PF_NTH;    // frames per tile

// Member row stride (words) of the shared tile for CW chunk slots per pair:
// with the staging lane map below, the eight stores of one step hit 32
// distinct banks (CW = 4: 8 c R = 8 c mod 32; CW = 2: 8 c R = 16 c mod 32).
template <int CW>
__host__ __device__ constexpr int pf_row() { return PF_NTH + (CW == 2 ? 2 : 1); }

// Stores the member word v of frame pair p in member row r (the row's word
// offset; -1: the station is in no group).
__device__ __forceinline__ void pf_put(uint32_t* xs, int r, int p, uint32_t v) {
  if (r >= 0) xs[r + p] = v;
}

// G groups; CW = 4 (at least 4 chunks of 8 stations per frame) or 2.
template <int G, int CW>
__global__ void __launch_bounds__(PF_NTH, 8) k_prebeam_pairs(
    const int8_t* __restrict__ x, const float2* __restrict__ w1, const int* __restrict__ member,
    const int* __restrict__ goff, int S, int K, int E, long long F, float scale,
    short2* __restrict__ y, unsigned long long* __restrict__ n_sat) {
  constexpr int R = pf_row<CW>();
  constexpr int PPW = 32 / CW;                                // pairs per warp and pass
  extern __shared__ float4 pf_smem[];
  float4* ws = pf_smem;                                       // [E] (wx, wx, wy, wy)
  int* mrow = reinterpret_cast<int*>(ws + E);                 // [S] row word offset or -1
  int* go = mrow + S;                                         // [G + 1]
  uint32_t* xs = reinterpret_cast<uint32_t*>(go + G + 1);    // [E][R]

  const int tile = blockIdx.x, k = blockIdx.y, pol = blockIdx.z;
  const int tid = threadIdx.x, fp = tid;
  const long long f0 = (long long)tile * PF_FT;
  const int nvalid = (int)min((long long)PF_FT, F - f0);
  for (int s = tid; s < S; s += PF_NTH) mrow[s] = -1;
  for (int g = tid; g <= G; g += PF_NTH) go[g] = goff[g];
  for (int e = tid; e < E; e += PF_NTH) {
    const float2 w = w1[(long long)k * E + e];
    ws[e] = make_float4(w.x, w.x, w.y, w.y);
  }
  __syncthreads();
  for (int e = tid; e < E; e += PF_NTH) mrow[member[e]] = e * R;
  __syncthreads();

  // Staging: frame pair p = 2 frames = 2 nq chunks of 16 bytes (frame a's nq,
  // then frame b's; chunk c holds stations 8c .. 8c + 7).  A lane takes chunk
  // slot cl of pair pl of its warp's PPW pairs, i.e. chunks c = cl, cl + CW,
  // ... of frames a and b: one load request covers PPW runs of 16 CW bytes,
  // and its samples go to the member rows as one word per station holding
  // (a.re, a.im, b.re, b.im).  Frames past the block end read as zero and are
  // never written.
  const int nq = S >> 3;
  const int lane = tid & 31, warp = tid >> 5;
  const int pl = lane / CW, cl = lane % CW;
  const uint4* xt = reinterpret_cast<const uint4*>(x + 2 * (((long long)pol * K + k) * F + f0) * S);
  const uint32_t m = 0x80808080u;                             // bytes offset by 128
#pragma unroll 2
  for (int pass = 0; pass < CW; ++pass) {
    const int p = warp * PPW + pl + pass * 4 * PPW;
    const bool va = 2 * p < nvalid, vb = 2 * p + 1 < nvalid;
    const uint4* xp = xt + (long long)p * 2 * nq;
    for (int c0 = cl; c0 < nq; c0 += 2 * CW) {
      uint4 a[2], b[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = c0 + u * CW;
        a[u] = make_uint4(0u, 0u, 0u, 0u);
        b[u] = a[u];
        if (c < nq) {
          if (va) a[u] = __ldg(xp + c);
          if (vb) b[u] = __ldg(xp + nq + c);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = c0 + u * CW;
        if (c >= nq) break;
        const int4 r0 = *reinterpret_cast<const int4*>(mrow + 8 * c);
        const int4 r1 = *reinterpret_cast<const int4*>(mrow + 8 * c + 4);
        pf_put(xs, r0.x, p, __byte_perm(a[u].x, b[u].x, 0x5410) ^ m);
        pf_put(xs, r0.y, p, __byte_perm(a[u].x, b[u].x, 0x7632) ^ m);
        pf_put(xs, r0.z, p, __byte_perm(a[u].y, b[u].y, 0x5410) ^ m);
        pf_put(xs, r0.w, p, __byte_perm(a[u].y, b[u].y, 0x7632) ^ m);
        pf_put(xs, r1.x, p, __byte_perm(a[u].z, b[u].z, 0x5410) ^ m);
        pf_put(xs, r1.y, p, __byte_perm(a[u].z, b[u].z, 0x7632) ^ m);
        pf_put(xs, r1.z, p, __byte_perm(a[u].w, b[u].w, 0x5410) ^ m);
        pf_put(xs, r1.w, p, __byte_perm(a[u].w, b[u].w, 0x7632) ^ m);
      }
    }
  }
  __syncthreads();
  const bool va = 2 * fp < nvalid, vb = 2 * fp + 1 < nvalid;

  // an unsigned byte u lands in the low mantissa bits of 2^23: the float is
  // 2^23 + u, and 2^23 + 128 + q = 2^23 + u recovers the sample q exactly
  const float2 boff = make_float2(-(8388608.0f + 128.0f), -(8388608.0f + 128.0f));
  const float2 sc = make_float2(scale, scale);
  const float2 rnd = make_float2(12582912.0f, 12582912.0f);   // 1.5 * 2^23
  uint32_t ca[G], cb[G];                                      // codes of frames a, b
  int sat = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    // re = sum wx A - sum wy B, im = sum wx B + sum wy A over the members,
    // A = (re of a, re of b), B = (im of a, im of b)
    float2 r1 = make_float2(0.f, 0.f), r2 = r1, im = r1;
    const int e1 = go[g + 1];
#pragma unroll 2
    for (int e = go[g]; e < e1; ++e) {
      const float4 w = ws[e];                                 // broadcast
      const uint32_t u = xs[e * R + fp];
      const float2 A = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7650)),
                                              __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7652))),
                                  boff);
      const float2 B = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7651)),
                                              __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7653))),
                                  boff);
      const float2 wx = make_float2(w.x, w.y), wy = make_float2(w.z, w.w);
      r1 = __ffma2_rn(wx, A, r1);
      r2 = __ffma2_rn(wy, B, r2);
      im = __ffma2_rn(wx, B, im);
      im = __ffma2_rn(wy, A, im);
    }
    float2 vr = __fmul2_rn(__fadd2_rn(r1, make_float2(-r2.x, -r2.y)), sc);
    float2 vi = __fmul2_rn(im, sc);
    const float mx = fmaxf(fmaxf(fabsf(vr.x), fabsf(vr.y)), fmaxf(fabsf(vi.x), fabsf(vi.y)));
    if (mx >= 32767.5f) {
      // saturation (rare): count the codes of valid frames, clamp all four
      sat += va ? (fabsf(vr.x) >= 32767.5f) + (fabsf(vi.x) >= 32767.5f) : 0;
      sat += vb ? (fabsf(vr.y) >= 32767.5f) + (fabsf(vi.y) >= 32767.5f) : 0;
      vr = make_float2(fminf(fmaxf(vr.x, -32767.f), 32767.f), fminf(fmaxf(vr.y, -32767.f), 32767.f));
      vi = make_float2(fminf(fmaxf(vi.x, -32767.f), 32767.f), fminf(fmaxf(vi.y, -32767.f), 32767.f));
    }
    // |v| <= 32767: v + 1.5 * 2^23 rounds v to an integer (half to even) whose
    // two's-complement low 16 bits are the float's low 16 bits
    const float2 qr = __fadd2_rn(vr, rnd), qi = __fadd2_rn(vi, rnd);
    ca[g] = __byte_perm(__float_as_uint(qr.x), __float_as_uint(qi.x), 0x5410);
    cb[g] = __byte_perm(__float_as_uint(qr.y), __float_as_uint(qi.y), 0x5410);
  }
  const int wsat = __reduce_add_sync(0xffffffffu, sat);
  if ((threadIdx.x & 31) == 0 && wsat) atomicAdd(n_sat, (unsigned long long)wsat);
  // [frame][group] codes: frames a and b are 2 G contiguous words (16-byte aligned)
  uint4* yo = reinterpret_cast<uint4*>(y + (((long long)pol * K + k) * F + f0 + 2 * fp) * G);
  if (va) {
#pragma unroll
    for (int i = 0; i < G / 4; ++i) yo[i] = make_uint4(ca[4 * i], ca[4 * i + 1], ca[4 * i + 2], ca[4 * i + 3]);
  }
  if (vb) {
#pragma unroll
    for (int i = 0; i < G / 4; ++i)
      yo[G / 4 + i] = make_uint4(cb[4 * i], cb[4 * i + 1], cb[4 * i + 2], cb[4 * i + 3]);
  }
}

// w1[k][e] = exp(-2 pi i nu_k ((r_s - r_g) . s_g) / c): the argument in FP64
// cycles, reduced to [-1/2, 1/2] before the FP32 sincospif
__global__ void k_prebeam_weights(const double* __restrict__ rel, const double* __restrict__ dir,
                                  int K, int E, int first_bin, float2* __restrict__ w1) {
  const long long total = (long long)K * E;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i % E);
    const int k = (int)(i / E);
    const double nu = kNu0 + (double)(first_bin + k) * (kFs / kM);
    const double dot = rel[3 * e] * dir[3 * e] + rel[3 * e + 1] * dir[3 * e + 1] +
                       rel[3 * e + 2] * dir[3 * e + 2];
    const double cyc = nu * dot / kC;
    const double r = cyc - rint(cyc);
    float sn, cs;
    sincospif(2.0f * (float)r, &sn, &cs);
    w1[i] = make_float2(cs, -sn);
  }
}

size_t prebeam_smem(const lp_prebeam& pb) {
  const size_t t2 = pb.input_dtype == LP_INPUT_INT8 ? sizeof(char2) : sizeof(short2);
  return sizeof(float4) * pb.E + t2 * (size_t)pb.S * PB_FTP +
         sizeof(short2) * (size_t)pb.G * PB_YP + sizeof(int) * (size_t)(pb.G + 1);
}

size_t prebeam_pairs_smem(const lp_prebeam& pb) {
  return sizeof(float4) * pb.E + sizeof(int) * ((size_t)pb.S + pb.G + 1) +
         sizeof(uint32_t) * (size_t)pb.E * pf_row<2>();
}

// The frame-pair kernel's shape conditions (the 16-byte alignment of the
// input and output pointers is checked per call).
bool prebeam_pairs_shape(const lp_prebeam& pb) {
  return pb.input_dtype == LP_INPUT_INT8 && pb.S % 8 == 0 && pb.S >= 16 &&
         (pb.G == 4 || pb.G == 8 || pb.G == 16) && prebeam_pairs_smem(pb) <= 227 * 1024;
}

const void* prebeam_pairs_kernel(int G, int S) {
  if (S >= 32)
    return G == 4 ? (const void*)k_prebeam_pairs<4, 4>
                  : G == 8 ? (const void*)k_prebeam_pairs<8, 4> : (const void*)k_prebeam_pairs<16, 4>;
  return G == 4 ? (const void*)k_prebeam_pairs<4, 2>
                : G == 8 ? (const void*)k_prebeam_pairs<8, 2> : (const void*)k_prebeam_pairs<16, 2>;
}

lp_status pb_fail(lp_prebeam* pb, lp_status st, const char* fmt, ...) {
  if (pb) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pb->err = buf;
  }
  return st;
}

#define PB_CUDA(pb, call)                                                            \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return pb_fail(pb, LP_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                     __FILE__, __LINE__);                                            \
  } while (0)

lp_status pb_set_device(lp_prebeam* pb) {
  int cur = -1;
  PB_CUDA(pb, cudaGetDevice(&cur));
  if (cur != pb->device) PB_CUDA(pb, cudaSetDevice(pb->device));
  return LP_OK;
}

// Carve the workspace (sized for every station in a group, so later
// lp_prebeam_set_groups calls never need more); base == nullptr: size only.
size_t pb_carve(lp_prebeam& pb, char* base) {
  size_t off = 0;
  auto take = [&](size_t n) -> char* {
    off = (off + 255) / 256 * 256;
    char* p = base ? base + off : nullptr;
    off += n;
    return p;
  };
  const int S = pb.S, G = pb.G;
  pb.w1 = (float2*)take(sizeof(float2) * (size_t)pb.K * S);
  pb.rel = (double*)take(sizeof(double) * 3 * (size_t)S);
  pb.mdir = (double*)take(sizeof(double) * 3 * (size_t)S);
  pb.member = (int*)take(sizeof(int) * S);
  pb.goff = (int*)take(sizeof(int) * (G + 1));
  pb.n_sat = (unsigned long long*)take(sizeof(unsigned long long));
  return (off + 255) / 256 * 256;
}

lp_status pb_device_pointer(lp_prebeam* pb, const void* ptr, const char* what) {
  cudaPointerAttributes attr;
  PB_CUDA(pb, cudaPointerGetAttributes(&attr, ptr));
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return pb_fail(pb, LP_ERR_ARG, "%s is not device memory", what);
  if (attr.device != pb->device)
    return pb_fail(pb, LP_ERR_ARG, "%s lives on device %d, the groups on %d", what, attr.device,
                   pb->device);
  return LP_OK;
}

}  // namespace
}  // namespace lp

extern "C" {

lp_status lp_prebeam_create(lp_prebeam** out, int stations, int pols, int subbands,
                            int64_t block_len, int groups, int first_bin, int input_dtype) {
  if (!out) return LP_ERR_ARG;
  *out = nullptr;
  if (stations < 1 || stations > 4096 || (pols != 1 && pols != 2) || subbands < 1 ||
      block_len < 1 || groups < 1 || groups > stations || groups > 4096)
    return LP_ERR_ARG;
  if (first_bin < 1 || first_bin + subbands > lp::kBins) return LP_ERR_ARG;
  if (input_dtype != LP_INPUT_INT8 && input_dtype != LP_INPUT_INT16) return LP_ERR_ARG;
  lp_prebeam* pb = new (std::nothrow) lp_prebeam;
  if (!pb) return LP_ERR_OOM;
  pb->S = stations;
  pb->P = pols;
  pb->K = subbands;
  pb->F = block_len;
  pb->G = groups;
  pb->first_bin = first_bin;
  pb->input_dtype = input_dtype;
  *out = pb;
  return LP_OK;
}

lp_status lp_prebeam_workspace_bytes(const lp_prebeam* pb, size_t* bytes) {
  if (!pb || !bytes) return LP_ERR_ARG;
  lp_prebeam tmp;
  tmp.S = pb->S;
  tmp.K = pb->K;
  tmp.G = pb->G;
  *bytes = lp::pb_carve(tmp, nullptr);
  return LP_OK;
}

lp_status lp_prebeam_bind_workspace(lp_prebeam* pb, void* dev, size_t bytes, void* stream) {
  using namespace lp;
  if (!pb) return LP_ERR_ARG;
  if (pb->mem) return pb_fail(pb, LP_ERR_STATE, "a workspace is already bound");
  if (!dev || (reinterpret_cast<uintptr_t>(dev) & 255u))
    return pb_fail(pb, LP_ERR_ARG, "workspace must be a 256-byte aligned device pointer");
  size_t need = 0;
  lp_prebeam_workspace_bytes(pb, &need);
  if (bytes < need) return pb_fail(pb, LP_ERR_OOM, "workspace %zu bytes < %zu needed", bytes, need);
  cudaPointerAttributes attr;
  PB_CUDA(pb, cudaPointerGetAttributes(&attr, dev));
  if (attr.type != cudaMemoryTypeDevice)
    return pb_fail(pb, LP_ERR_ARG, "workspace is not device memory");
  pb->device = attr.device;
  if (pb_set_device(pb) != LP_OK) return LP_ERR_CUDA;
  pb->mem = dev;
  pb_carve(*pb, static_cast<char*>(dev));
  PB_CUDA(pb, cudaMemsetAsync(pb->n_sat, 0, sizeof(unsigned long long),
                              static_cast<cudaStream_t>(stream)));
  pb->last_stream = static_cast<cudaStream_t>(stream);
  return LP_OK;
}

lp_status lp_prebeam_set_groups(lp_prebeam* pb, const int32_t* group_of_station,
                                const double* station_enu, const double* group_dir,
                                void* stream) {
  using namespace lp;
  if (!pb) return LP_ERR_ARG;
  if (!group_of_station || !station_enu || !group_dir)
    return pb_fail(pb, LP_ERR_ARG, "null group table, positions or directions");
  const int S = pb->S, G = pb->G;
  std::vector<int> count(G, 0);
  for (int s = 0; s < S; ++s) {
    const int g = group_of_station[s];
    if (g < -1 || g >= G) return pb_fail(pb, LP_ERR_ARG, "station %d: group %d not in [-1, %d)", s, g, G);
    if (g >= 0) count[g] += 1;
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(station_enu[3 * s + c]))
        return pb_fail(pb, LP_ERR_ARG, "station %d position not finite", s);
  }
  for (int g = 0; g < G; ++g) {
    if (!count[g]) return pb_fail(pb, LP_ERR_ARG, "group %d has no station", g);
    const double* d = group_dir + 3 * g;
    const double n2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(std::fabs(n2 - 1.0) < 1e-6))
      return pb_fail(pb, LP_ERR_ARG, "direction of group %d is not a unit vector", g);
  }
  // phase centres (member means) and the member list sorted by group
  std::vector<double> centres(3 * (size_t)G, 0.0);
  for (int s = 0; s < S; ++s) {
    const int g = group_of_station[s];
    if (g < 0) continue;
    for (int c = 0; c < 3; ++c) centres[3 * g + c] += station_enu[3 * s + c];
  }
  for (int g = 0; g < G; ++g)
    for (int c = 0; c < 3; ++c) centres[3 * g + c] /= count[g];
  std::vector<int> member, goff(G + 1, 0);
  std::vector<double> rel, mdir;
  for (int g = 0; g < G; ++g) {
    goff[g] = (int)member.size();
    for (int s = 0; s < S; ++s) {
      if (group_of_station[s] != g) continue;
      member.push_back(s);
      for (int c = 0; c < 3; ++c) {
        rel.push_back(station_enu[3 * s + c] - centres[3 * g + c]);
        mdir.push_back(group_dir[3 * g + c]);
      }
    }
  }
  goff[G] = (int)member.size();
  const int E = goff[G];
  if (!pb->mem) return pb_fail(pb, LP_ERR_STATE, "bind a workspace first");

  if (pb_set_device(pb) != LP_OK) return LP_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pb->E = E;
  // pageable host memory: the copies are complete for the host on return
  PB_CUDA(pb, cudaMemcpyAsync(pb->member, member.data(), sizeof(int) * E, cudaMemcpyHostToDevice, s));
  PB_CUDA(pb, cudaMemcpyAsync(pb->goff, goff.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, s));
  PB_CUDA(pb, cudaMemcpyAsync(pb->rel, rel.data(), sizeof(double) * 3 * E, cudaMemcpyHostToDevice, s));
  PB_CUDA(pb, cudaMemcpyAsync(pb->mdir, mdir.data(), sizeof(double) * 3 * E, cudaMemcpyHostToDevice, s));
  const long long total = (long long)pb->K * E;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  k_prebeam_weights<<<blocks, 256, 0, s>>>(pb->rel, pb->mdir, pb->K, E, pb->first_bin, pb->w1);
  PB_CUDA(pb, cudaGetLastError());
  const int smem = (int)prebeam_smem(*pb);
  if (smem > 227 * 1024) return pb_fail(pb, LP_ERR_ARG, "too many stations for one tile");
  if (pb->input_dtype == LP_INPUT_INT8)
    PB_CUDA(pb, raise_smem_limit((const void*)k_prebeam<char2>, (size_t)smem));
  else
    PB_CUDA(pb, raise_smem_limit((const void*)k_prebeam<short2>, (size_t)smem));
  if (prebeam_pairs_shape(*pb))
    PB_CUDA(pb, raise_smem_limit(prebeam_pairs_kernel(G, S), prebeam_pairs_smem(*pb)));
  pb->centres = centres;
  pb->last_stream = s;
  pb->groups_set = true;
  return LP_OK;
}

lp_status lp_prebeam_group_centres(lp_prebeam* pb, double* centre_enu) {
  if (!pb || !centre_enu) return LP_ERR_ARG;
  if (!pb->groups_set) return lp::pb_fail(pb, LP_ERR_STATE, "lp_prebeam_set_groups first");
  for (size_t i = 0; i < pb->centres.size(); ++i) centre_enu[i] = pb->centres[i];
  return LP_OK;
}

lp_status lp_prebeam_run(lp_prebeam* pb, const void* x, void* y, float scale, void* stream) {
  using namespace lp;
  if (!pb) return LP_ERR_ARG;
  if (!pb->groups_set) return pb_fail(pb, LP_ERR_STATE, "lp_prebeam_set_groups first");
  if (!x || !y) return pb_fail(pb, LP_ERR_ARG, "null input or output");
  if (!(scale > 0.f) || !std::isfinite(scale))
    return pb_fail(pb, LP_ERR_ARG, "scale must be positive and finite");
  if (pb_set_device(pb) != LP_OK) return LP_ERR_CUDA;
  if (lp_status st = pb_device_pointer(pb, x, "input")) return st;
  if (lp_status st = pb_device_pointer(pb, y, "output")) return st;
  const size_t t2 = pb->input_dtype == LP_INPUT_INT8 ? 2 : 4;
  if (reinterpret_cast<uintptr_t>(x) % t2 || reinterpret_cast<uintptr_t>(y) % 4)
    return pb_fail(pb, LP_ERR_ARG, "input must be %zu-byte and output 4-byte aligned", t2);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dim3 grid((unsigned)((pb->F + PB_FT - 1) / PB_FT), pb->K, pb->P);
  const size_t smem = prebeam_smem(*pb);
  // 16-byte chunk reads when every (pol, subband) slab starts 16-byte aligned
  // (tiles then do too: 256 frames of S samples of 2 or 4 bytes)
  const int vec = reinterpret_cast<uintptr_t>(x) % 16 == 0 && (pb->F * pb->S * t2) % 16 == 0;
  if (vec && reinterpret_cast<uintptr_t>(y) % 16 == 0 && prebeam_pairs_shape(*pb)) {
    const dim3 pgrid((unsigned)((pb->F + PF_FT - 1) / PF_FT), pb->K, pb->P);
    const size_t psmem = prebeam_pairs_smem(*pb);
    const int8_t* x8 = static_cast<const int8_t*>(x);
    short2* y2 = static_cast<short2*>(y);
    const void* kern = prebeam_pairs_kernel(pb->G, pb->S);
    void* args[] = {(void*)&x8, (void*)&pb->w1, (void*)&pb->member, (void*)&pb->goff,
                    (void*)&pb->S, (void*)&pb->K, (void*)&pb->E, (void*)&pb->F,
                    (void*)&scale, (void*)&y2, (void*)&pb->n_sat};
    PB_CUDA(pb, cudaLaunchKernel(kern, pgrid, dim3(PF_NTH), args, psmem, s));
  } else if (pb->input_dtype == LP_INPUT_INT8)
    k_prebeam<char2><<<grid, PB_NTH, smem, s>>>(static_cast<const char2*>(x), pb->w1, pb->member,
                                                pb->goff, pb->S, pb->K, pb->G, pb->E, pb->F,
                                                scale, vec, static_cast<short2*>(y), pb->n_sat);
  else
    k_prebeam<short2><<<grid, PB_NTH, smem, s>>>(static_cast<const short2*>(x), pb->w1,
                                                 pb->member, pb->goff, pb->S, pb->K, pb->G,
                                                 pb->E, pb->F, scale, vec,
                                                 static_cast<short2*>(y), pb->n_sat);
  PB_CUDA(pb, cudaGetLastError());
  pb->last_stream = s;
  return LP_OK;
}

lp_status lp_prebeam_saturated(lp_prebeam* pb, int64_t* n) {
  using namespace lp;
  if (!pb || !n) return LP_ERR_ARG;
  *n = 0;
  if (!pb->mem) return LP_OK;
  if (pb_set_device(pb) != LP_OK) return LP_ERR_CUDA;
  PB_CUDA(pb, cudaStreamSynchronize(pb->last_stream));
  unsigned long long v = 0;
  PB_CUDA(pb, cudaMemcpy(&v, pb->n_sat, sizeof v, cudaMemcpyDeviceToHost));
  PB_CUDA(pb, cudaMemset(pb->n_sat, 0, sizeof v));
  *n = (int64_t)v;
  return LP_OK;
}

const char* lp_prebeam_last_error(const lp_prebeam* pb) {
  return pb ? pb->err.c_str() : "null preliminary-beam plan";
}

void lp_prebeam_destroy(lp_prebeam* pb) {
  delete pb;   // the workspace stays the caller's
}

}  // extern "C"
