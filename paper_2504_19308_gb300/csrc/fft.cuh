// Shared-memory Stockham FFTs for lengths N = 3^c 2^a (sm_103a).
//
// A CTA transforms S signals of length N that sit in shared memory, one after another,
// each padded by fpad() (one float2 every 16).  Passes are radix 3 for each factor 3, then
// radix 16, then one pass of radix 2, 4 or 8 for the remaining factor.  Each pass is the
// Stockham autosort step
// (Stockham 1966; the GPU formulation of Govindaraju et al., SC 2008):
//
//     for every butterfly j in [0, N/R):  m = j mod Ns
//         v[r] = x[j + r N/R] * w^(r m N/(Ns R)),  r = 0..R-1      (w = e^{-+2 pi i/N})
//         v    = DFT_R(v)
//         y[(j / Ns) Ns R + m + r Ns] = v[r]
//
// which leaves the result in natural order.  Loads of a pass complete (barrier) before
// its stores, so the same buffer is read and written.  Twiddles come from a table
// tw[m] = e^{-2 pi i m / N} built once per N in double precision and rounded to float; a
// butterfly reads the powers 1, 2, 4, 8 of its twiddle and multiplies out the others.
// Forward = unnormalised DFT (sign -); inverse = sign +, no 1/N (callers scale).
#pragma once
#include "common.cuh"

namespace amm {

// ----------------------------------------------------------------------------- DFT_R in registers
template <bool INV> AMM_DEV float2 mul_mi(float2 a) {  // a * (-i) forward, a * (+i) inverse
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV> AMM_DEV void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV> AMM_DEV void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  float2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// e^{-+2 pi i m / 16} for the twiddles inside DFT_16 / DFT_8 (cos/sin of multiples of pi/8).
#define AMM_C1 0.92387953251128674f  /* cos(pi/8) */
#define AMM_S1 0.38268343236508977f  /* sin(pi/8) */
#define AMM_R2 0.70710678118654752f  /* cos(pi/4) */

template <bool INV> AMM_DEV float2 w16mul(float2 a, int m) {
  float c, s;  // e^{-i m pi/8} = c - i s  (forward)
  switch (m & 15) {
    case 0: return a;
    case 1: c = AMM_C1; s = AMM_S1; break;
    case 2: c = AMM_R2; s = AMM_R2; break;
    case 3: c = AMM_S1; s = AMM_C1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 6: c = -AMM_R2; s = AMM_R2; break;
    case 9: c = -AMM_C1; s = -AMM_S1; break;
    default: c = 1.f; s = 0.f; break;  // not reached for the products n2*k1 used below
  }
  if (INV) s = -s;
  return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

template <bool INV> AMM_DEV void dft8(float2* v) {
  // X[k] = E[k] + w8^k O[k], X[k+4] = E[k] - w8^k O[k]; E/O = DFT_4 of even/odd samples.
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = w16mul<INV>(o1, 2);
  o2 = w16mul<INV>(o2, 4);
  o3 = w16mul<INV>(o3, 6);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <bool INV> AMM_DEV void dft16(float2* v) {
  // n = 4 n1 + n2, k = k1 + 4 k2:  X[k1 + 4 k2] = sum_n2 w16^(n2 k1) w4^(n2 k2) DFT4_n1(x[4 n1 + n2])[k1]
  float2 y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2], a3 = v[12 + n2];
    dft4<INV>(a0, a1, a2, a3);
    y[n2][0] = a0;
    y[n2][1] = w16mul<INV>(a1, n2);
    y[n2][2] = w16mul<INV>(a2, 2 * n2);
    y[n2][3] = w16mul<INV>(a3, 3 * n2);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a0 = y[0][k1], a1 = y[1][k1], a2 = y[2][k1], a3 = y[3][k1];
    dft4<INV>(a0, a1, a2, a3);
    v[k1] = a0; v[k1 + 4] = a1; v[k1 + 8] = a2; v[k1 + 12] = a3;
  }
}

// DFT_3: X[k] = sum_n x[n] e^{-+2 pi i n k / 3}; with s = x1 + x2, d = x1 - x2:
// X0 = x0 + s, X1,2 = x0 - s/2 -+ i (sqrt(3)/2) d  (forward; the inverse swaps the signs of i).
#define AMM_H3 0.86602540378443865f  /* sqrt(3) / 2 */
template <bool INV> AMM_DEV void dft3(float2& a0, float2& a1, float2& a2) {
  const float2 s = cadd(a1, a2), d = csub(a1, a2);
  const float2 m = make_float2(fmaf(-0.5f, s.x, a0.x), fmaf(-0.5f, s.y, a0.y));
  const float2 r = INV ? make_float2(-AMM_H3 * d.y, AMM_H3 * d.x) : make_float2(AMM_H3 * d.y, -AMM_H3 * d.x);
  a0 = cadd(a0, s);
  a1 = cadd(m, r);
  a2 = csub(m, r);
}

template <int R, bool INV> AMM_DEV void dft_r(float2* v) {
  if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else dft16<INV>(v);
}

// ----------------------------------------------------------------------------- twiddle powers
// w[r] = tw[r * base] (r = 1 .. R-1) for a butterfly of radix R, conjugated for INV.  The powers
// 1, 2, 4, 8 are read from the table and the others formed as products of at most three of them
// (w3 = w1 w2, w5 = w4 w1, ..., w15 = w8 (w4 w3)): four loads instead of fifteen through the L1
// pipe for R = 16, at a cost of a few ulp in the formed twiddles.
template <int R, bool INV>
AMM_DEV void twiddle_powers(const float2* __restrict__ tw, int base, float2* w) {
  auto ld = [&](int r) {
    float2 v = __ldg(tw + r * base);
    if (INV) v.y = -v.y;
    return v;
  };
  if constexpr (R <= 3) {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = ld(r);
  } else {
    w[1] = ld(1);
    w[2] = ld(2);
    w[3] = cmul(w[1], w[2]);
    if constexpr (R >= 8) {
      w[4] = ld(4);
#pragma unroll
      for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
    }
    if constexpr (R >= 16) {
      w[8] = ld(8);
#pragma unroll
      for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
    }
  }
}

// ----------------------------------------------------------------------------- one Stockham pass
// S signals of length N, signal s at buf + s * fft_padded_len(N), NT threads cooperating.
// UNPAD_OUT: store the pass's output at plain (unpadded) indices.  Used for the last pass of a
// transform whose result is read with arbitrary shifts (the stores of a last pass are contiguous
// across threads, so they stay conflict-free without padding).
template <int N, int R, int NS, int S, int NT, bool INV, bool UNPAD_OUT = false>
AMM_DEV void stockham_pass(float2* buf, const float2* __restrict__ tw) {
  constexpr int NB = N / R;
  constexpr int TOT = NB * S;
  constexpr int PER = (TOT + NT - 1) / NT;
  constexpr int TWS = N / (NS * R);  // twiddle index stride
  constexpr int LD = fft_padded_len(N);
  float2 v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if (PER * NT == TOT || b < TOT) {
      const int s = b / NB, j = b % NB;
      const float2* x = buf + s * LD;
      const int m = j % NS;
      float2 w[R];
      if (NS > 1) twiddle_powers<R, INV>(tw, m * TWS, w);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 a = x[fpad(j + r * NB)];
        if (NS > 1 && r > 0) a = cmul(a, w[r]);
        v[i][r] = a;
      }
      dft_r<R, INV>(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = threadIdx.x + i * NT;
    if (PER * NT == TOT || b < TOT) {
      const int s = b / NB, j = b % NB;
      float2* y = buf + s * LD;
      const int m = j % NS;
      const int base = (j / NS) * NS * R + m;
#pragma unroll
      for (int r = 0; r < R; ++r) y[UNPAD_OUT ? base + r * NS : fpad(base + r * NS)] = v[i][r];
    }
  }
  __syncthreads();
}

template <int N, int NS, int S, int NT, bool INV, bool UNPAD_LAST>
struct FftPasses {
  static AMM_DEV void run(float2* buf, const float2* __restrict__ tw) {
    constexpr int LEFT = N / NS;
    constexpr int R = (LEFT % 3 == 0) ? 3 : (LEFT >= 16) ? 16 : LEFT;
    stockham_pass<N, R, NS, S, NT, INV, UNPAD_LAST && (NS * R == N)>(buf, tw);
    FftPasses<N, NS * R, S, NT, INV, UNPAD_LAST>::run(buf, tw);
  }
};
template <int N, int S, int NT, bool INV, bool UNPAD_LAST>
struct FftPasses<N, N, S, NT, INV, UNPAD_LAST> {
  static AMM_DEV void run(float2*, const float2* __restrict__) {}
};

// Transform S padded signals in place.  Must be called by all NT threads; ends with a barrier.
// With UNPAD_LAST the result is left at plain indices (signal s still starts at s * padded len).
template <int N, int S, int NT, bool INV, bool UNPAD_LAST = false>
AMM_DEV void fft_smem(float2* buf, const float2* __restrict__ tw) {
  static_assert(fft_len_ok(N) && N >= 2, "N = 3^c 2^a");
  FftPasses<N, 1, S, NT, INV, UNPAD_LAST>::run(buf, tw);
}

}  // namespace amm
