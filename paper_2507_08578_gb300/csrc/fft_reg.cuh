// Register-resident DFT codelets and a two-level pencil FFT for the local-potential path.
//
// A pencil of length N = A*B is transformed by a group of L = max(A, B) lanes:
//   stage 1: lane j < B holds x[j + B*i] (i < A), does a DFT of size A in registers,
//            multiplies output k1 by w_N^{j*k1} and stores it to per-pencil scratch;
//   stage 2: lane k1 < A reads the B values of its column, does a DFT of size B in registers
//            and holds X[k1 + A*k2] (k2 < B).
// (X[k1 + A k2] = sum_j w_B^{j k2} w_N^{j k1} sum_i x[j + B i] w_A^{i k1}, the two-factor
// Cooley-Tukey split.)  Only one exchange through shared memory per transform.
// Codelets of size 2..16 ({2,3,4,5} and products) are fully unrolled with compile-time
// twiddle constants; their cos/sin values are Taylor series evaluated by the compiler.
#pragma once

#include <type_traits>

namespace kss {
namespace fftr {

// floor(t / d) for 0 <= t < 2^22 and d >= 1 by one multiply with the float reciprocal of d (the
// index arithmetic of the CTA-wide task loops, whose divisors are runtime window sizes): (t + 1/2)/d
// lies at least 1/(2d) from an integer, and the roundings of the reciprocal and of the product
// move it by at most 2^-23 (t + 1/2)/d < 1/(2d), so truncation gives the exact quotient.
struct FastDiv {
  float r;
  __device__ __forceinline__ explicit FastDiv(int d) : r(1.0f / (float)d) {}
  __device__ __forceinline__ int operator()(int t) const { return __float2int_rz(((float)t + 0.5f) * r); }
};
// (lo + u) mod n for lo in (-n, n) and 0 <= u < n (a window index to a box coordinate).
__device__ __forceinline__ int wrap_add(int lo, int u, int n) {
  int y = lo + u;
  if (y < 0) y += n;
  if (y >= n) y -= n;
  return y;
}

// ---- compile-time trig: cos/sin(2 pi m / n) --------------------------------------------------
__host__ __device__ constexpr double taylor_sin(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// Reduce to a quadrant with integer arithmetic, then a Taylor series on [0, pi/2).
__host__ __device__ constexpr double kcos(int m, int n) {
  m %= n;
  if (m < 0) m += n;
  const int q = (4 * m) / n;
  const int r = 4 * m - q * n;
  const double phi = 1.5707963267948966 * (double)r / (double)n;
  return q == 0 ? taylor_cos(phi) : q == 1 ? -taylor_sin(phi) : q == 2 ? -taylor_cos(phi) : taylor_sin(phi);
}
__host__ __device__ constexpr double ksin(int m, int n) {
  m %= n;
  if (m < 0) m += n;
  const int q = (4 * m) / n;
  const int r = 4 * m - q * n;
  const double phi = 1.5707963267948966 * (double)r / (double)n;
  return q == 0 ? taylor_sin(phi) : q == 1 ? taylor_cos(phi) : q == 2 ? -taylor_sin(phi) : -taylor_cos(phi);
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

template <typename C> __device__ __forceinline__ C add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C mul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// multiply by s*i for s = +-1: sign flips only (no multiplication)
template <typename C, typename T> __device__ __forceinline__ C muli(C a, T s) {
  C r;
  if (s > (T)0) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}
// multiply by s*m*i for s = +-1 and a constant m > 0
template <typename C, typename T> __device__ __forceinline__ C muli_m(C a, T s, T m) {
  const T ms = s > (T)0 ? m : -m;
  C r;
  r.x = -ms * a.y;
  r.y = ms * a.x;
  return r;
}

__host__ __device__ constexpr int first_factor(int n) { return n % 4 == 0 && n != 4 ? 4 : n % 2 == 0 && n != 2 ? 2 : n % 3 == 0 && n != 3 ? 3 : n % 5 == 0 && n != 5 ? 5 : n; }

// y_q = sum_t v_t exp(s * 2 pi i t q / N), natural order in and out.
template <int N, typename C, typename T> __device__ __forceinline__ void rdft(C* v, T s);

template <int N, typename C, typename T>
__device__ __forceinline__ void rdft_base(C* v, T s) {
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    const C a = v[0], b = v[1];
    v[0] = add(a, b);
    v[1] = sub(a, b);
  } else if constexpr (N == 3) {
    const T h = (T)0.5, s3 = (T)0.86602540378443864676;
    const C t1 = add(v[1], v[2]);
    C t2;
    t2.x = v[0].x - h * t1.x;
    t2.y = v[0].y - h * t1.y;
    const C t3 = muli_m(sub(v[1], v[2]), s, s3);
    v[0] = add(v[0], t1);
    v[1] = add(t2, t3);
    v[2] = sub(t2, t3);
  } else if constexpr (N == 4) {
    const C a = add(v[0], v[2]), b = sub(v[0], v[2]);
    const C c = add(v[1], v[3]), d = muli(sub(v[1], v[3]), s);
    v[0] = add(a, c);
    v[2] = sub(a, c);
    v[1] = add(b, d);
    v[3] = sub(b, d);
  } else if constexpr (N == 5) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    const C a1 = add(v[1], v[4]), a2 = add(v[2], v[3]);
    const C b1 = sub(v[1], v[4]), b2 = sub(v[2], v[3]);
    C r1, r2, w1, w2;
    r1.x = v[0].x + c1 * a1.x + c2 * a2.x;
    r1.y = v[0].y + c1 * a1.y + c2 * a2.y;
    r2.x = v[0].x + c2 * a1.x + c1 * a2.x;
    r2.y = v[0].y + c2 * a1.y + c1 * a2.y;
    w1.x = s1 * b1.x + s2 * b2.x;
    w1.y = s1 * b1.y + s2 * b2.y;
    w2.x = s2 * b1.x - s1 * b2.x;
    w2.y = s2 * b1.y - s1 * b2.y;
    const C i1 = muli(w1, s), i2 = muli(w2, s);
    v[0] = add(v[0], add(a1, a2));
    v[1] = add(r1, i1);
    v[4] = sub(r1, i1);
    v[2] = add(r2, i2);
    v[3] = sub(r2, i2);
  }
}

// Composite N = P * Q: DFT-P over i of x[j + Q i], twiddle w_N^{j k1}, DFT-Q over j.
template <int N, typename C, typename T>
__device__ __forceinline__ void rdft_split(C* v, T s) {
  constexpr int P = first_factor(N);
  constexpr int Q = N / P;
  C t[Q][P];
  static_for<0, Q>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    static_for<0, P>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      t[j][i] = v[j + Q * i];
    });
    rdft<P>(t[j], s);
    static_for<1, P>([&](auto kc) {
      constexpr int k1 = decltype(kc)::value;
      if constexpr ((j * k1) % N != 0) {
        constexpr double wc = kcos(j * k1, N), ws = ksin(j * k1, N);
        if constexpr (wc == 0.0 && (ws == 1.0 || ws == -1.0)) {
          t[j][k1] = muli(t[j][k1], ws > 0.0 ? s : -s);  // w = +-i
        } else if constexpr (ws == 0.0 && wc == -1.0) {
          t[j][k1].x = -t[j][k1].x;  // w = -1
          t[j][k1].y = -t[j][k1].y;
        } else {
          C w;
          w.x = (T)wc;
          w.y = s > (T)0 ? (T)ws : -(T)ws;
          t[j][k1] = mul(t[j][k1], w);
        }
      }
    });
  });
  static_for<0, P>([&](auto kc) {
    constexpr int k1 = decltype(kc)::value;
    C u[Q];
    static_for<0, Q>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      u[j] = t[j][k1];
    });
    rdft<Q>(u, s);
    static_for<0, Q>([&](auto qc) {
      constexpr int k2 = decltype(qc)::value;
      v[k1 + P * k2] = u[k2];
    });
  });
}

template <int N, typename C, typename T>
__device__ __forceinline__ void rdft(C* v, T s) {
  if constexpr (N <= 5 && N != 4) rdft_base<N>(v, s);
  else if constexpr (N == 4) rdft_base<4>(v, s);
  else rdft_split<N>(v, s);
}

// ---- pruned transforms ---------------------------------------------------------------------------
// rdft_m<N, MIN, MOUT>: y_q = sum_{t in MIN} v_t w^{s t q} for every q in MOUT (bit masks over
// 0..N-1); inputs outside MIN are taken as zero (never read), outputs outside MOUT are left
// unspecified.  The composite form follows rdft_split step for step (same factors, twiddles and
// order), skipping the sub-transforms whose inputs are all zero, the twiddles and second-level
// transforms no needed output depends on, and, in the base transforms, every term of a zero input
// or an unneeded output; with full masks it performs exactly the operations of rdft.
template <int N> __host__ __device__ constexpr unsigned full_mask() { return N >= 32 ? 0xffffffffu : ((1u << N) - 1u); }
__host__ __device__ constexpr int popc(unsigned m) { int c = 0; for (; m; m &= m - 1) ++c; return c; }
__host__ __device__ constexpr int lowbit(unsigned m) { int i = 0; while (!(m >> i & 1u)) ++i; return i; }

// a * w^{E} with w = exp(s 2 pi i / N), compile-time E: the trivial factors without multiplies
template <int E, int N, typename C, typename T>
__device__ __forceinline__ C twiddle_c(C a, T s) {
  constexpr int e = ((E % N) + N) % N;
  if constexpr (e == 0) {
    return a;
  } else {
    constexpr double wc = kcos(e, N), ws = ksin(e, N);
    if constexpr (wc == 0.0 && (ws == 1.0 || ws == -1.0)) {
      return muli(a, ws > 0.0 ? s : -s);
    } else if constexpr (ws == 0.0 && wc == -1.0) {
      C r;
      r.x = -a.x;
      r.y = -a.y;
      return r;
    } else {
      C w;
      w.x = (T)wc;
      w.y = s > (T)0 ? (T)ws : -(T)ws;
      return mul(a, w);
    }
  }
}
template <int E, int N> __host__ __device__ constexpr int twiddle_cost() {
  constexpr int e = ((E % N) + N) % N;
  if constexpr (e == 0) return 0;
  else if constexpr ((kcos(e, N) == 0.0 && (ksin(e, N) == 1.0 || ksin(e, N) == -1.0)) ||
                     (ksin(e, N) == 0.0 && kcos(e, N) == -1.0)) return 0;
  else return 6;
}
// real operations of the direct sums of a masked base transform, and of the full codelet
template <int N, unsigned MIN, unsigned MOUT> __host__ __device__ constexpr int direct_cost() {
  int c = 0;
  for (int q = 0; q < N; ++q) {
    if (!(MOUT >> q & 1u)) continue;
    int terms = 0;
    for (int t = 0; t < N; ++t) {
      if (!(MIN >> t & 1u)) continue;
      const int e = (t * q) % N;
      const bool triv = e == 0 || (kcos(e, N) == 0.0 && (ksin(e, N) == 1.0 || ksin(e, N) == -1.0)) ||
                        (ksin(e, N) == 0.0 && kcos(e, N) == -1.0);
      c += triv ? 0 : 6;
      ++terms;
    }
    c += 2 * (terms - 1);
  }
  return c;
}
template <int N> __host__ __device__ constexpr int codelet_cost() {
  return N == 2 ? 4 : N == 3 ? 16 : N == 4 ? 16 : N == 5 ? 44 : 1 << 20;
}

template <int N, unsigned MIN, unsigned MOUT, typename C, typename T>
__device__ __forceinline__ void rdft_m(C* v, T s);

template <int N, unsigned MIN, unsigned MOUT, typename C, typename T>
__device__ __forceinline__ void rdft_direct(C* v, T s) {
  constexpr int t0 = lowbit(MIN);
  C in[N];
  static_for<0, N>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    if constexpr (MIN >> t & 1u) in[t] = v[t];
  });
  static_for<0, N>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    if constexpr (MOUT >> q & 1u) {
      C acc = twiddle_c<t0 * q, N>(in[t0], s);
      static_for<t0 + 1, N>([&](auto tc) {
        constexpr int t = decltype(tc)::value;
        if constexpr (MIN >> t & 1u) acc = add(acc, twiddle_c<t * q, N>(in[t], s));
      });
      v[q] = acc;
    }
  });
}

template <int N, unsigned MIN, unsigned MOUT, typename C, typename T>
__device__ __forceinline__ void rdft_split_m(C* v, T s) {
  constexpr int P = first_factor(N);
  constexpr int Q = N / P;
  // first-level outputs k1 that some needed output k1 + P k2 depends on
  constexpr unsigned need1 = [] {
    unsigned m = 0;
    for (int k1 = 0; k1 < P; ++k1)
      for (int k2 = 0; k2 < Q; ++k2)
        if (MOUT >> (k1 + P * k2) & 1u) m |= 1u << k1;
    return m;
  }();
  // sub-transforms j with a nonzero input (the second level's input mask)
  constexpr unsigned jm = [] {
    unsigned m = 0;
    for (int j = 0; j < Q; ++j)
      for (int i = 0; i < P; ++i)
        if (MIN >> (j + Q * i) & 1u) m |= 1u << j;
    return m;
  }();
  C t[Q][P];
  static_for<0, Q>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    constexpr unsigned mj = [] {
      unsigned m = 0;
      for (int i = 0; i < P; ++i)
        if (MIN >> (j + Q * i) & 1u) m |= 1u << i;
      return m;
    }();
    if constexpr (mj != 0u) {
      static_for<0, P>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if constexpr (mj >> i & 1u) t[j][i] = v[j + Q * i];
      });
      rdft_m<P, mj, need1>(t[j], s);
      static_for<1, P>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        if constexpr ((need1 >> k1 & 1u) && (j * k1) % N != 0) t[j][k1] = twiddle_c<j * k1, N>(t[j][k1], s);
      });
    }
  });
  static_for<0, P>([&](auto kc) {
    constexpr int k1 = decltype(kc)::value;
    if constexpr (need1 >> k1 & 1u) {
      constexpr unsigned mo2 = [] {
        unsigned m = 0;
        for (int k2 = 0; k2 < Q; ++k2)
          if (MOUT >> (k1 + P * k2) & 1u) m |= 1u << k2;
        return m;
      }();
      C u[Q];
      static_for<0, Q>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if constexpr (jm >> j & 1u) u[j] = t[j][k1];
      });
      rdft_m<Q, jm, mo2>(u, s);
      static_for<0, Q>([&](auto qc) {
        constexpr int k2 = decltype(qc)::value;
        if constexpr (mo2 >> k2 & 1u) v[k1 + P * k2] = u[k2];
      });
    }
  });
}

template <int N, unsigned MIN, unsigned MOUT, typename C, typename T>
__device__ __forceinline__ void rdft_m(C* v, T s) {
  static_assert(MIN != 0u && MOUT != 0u, "empty pruned transform");
  constexpr unsigned F = full_mask<N>();
  if constexpr (N == 1) {
  } else if constexpr ((MIN & F) == F && (MOUT & F) == F) {
    rdft<N>(v, s);
  } else if constexpr (N <= 5) {
    if constexpr (direct_cost<N, MIN, MOUT>() < codelet_cost<N>()) {
      rdft_direct<N, MIN, MOUT>(v, s);
    } else {
      static_for<0, N>([&](auto tc) {  // the full codelet reads every input: zero the pruned ones
        constexpr int t = decltype(tc)::value;
        if constexpr (!(MIN >> t & 1u)) {
          v[t].x = (T)0;
          v[t].y = (T)0;
        }
      });
      rdft_base<N>(v, s);
    }
  } else {
    rdft_split_m<N, MIN, MOUT>(v, s);
  }
}
// Mask of the window pattern of a pruned stage: the first C and the last C of N positions.
template <int N, int C> __host__ __device__ constexpr unsigned edge_mask() {
  return C <= 0 || 2 * C >= N ? full_mask<N>() : (((1u << C) - 1u) | (((1u << C) - 1u) << (N - C)));
}

// Runtime size dispatch over the codelet set {1,2,3,4,5,6,8,9,10,12,15,16}.
template <typename C, typename T>
__device__ __forceinline__ void rdft_rt(int n, C* v, T s) {
  switch (n) {
    case 2: rdft<2>(v, s); break;
    case 3: rdft<3>(v, s); break;
    case 4: rdft<4>(v, s); break;
    case 5: rdft<5>(v, s); break;
    case 6: rdft<6>(v, s); break;
    case 8: rdft<8>(v, s); break;
    case 9: rdft<9>(v, s); break;
    case 10: rdft<10>(v, s); break;
    case 12: rdft<12>(v, s); break;
    case 15: rdft<15>(v, s); break;
    case 16: rdft<16>(v, s); break;
    default: break;  // n == 1
  }
}

constexpr int kMaxR = 16;

// Split of one pencil length for the two-level transform (host-chosen).
struct Split {
  int N, A, B, L, PP;  // N = A*B, L = max(A,B) lanes per pencil, PP pencils per warp
  int scr;             // scratch elements per pencil
};

}  // namespace fftr
}  // namespace kss
