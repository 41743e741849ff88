// Reverse-mode (adjoint) gradient of the EGARCH(K, I) log likelihood with
// respect to the transformed parameters theta, and the MALA mutation built on
// it.  The paper's M phase uses a Gaussian random walk; it notes that other
// Metropolis updates are possible (Section 3.3, "Metropolis steps").  The
// Langevin proposal theta* = theta + (1/2) Sigma grad + L z, Sigma = L L', with
// grad the gradient of the tempered log target, keeps the posterior invariant
// through the Metropolis-Hastings correction q(theta | theta*) / q(theta* | theta).
//
// Forward recursion in natural units (one particle, t = 1..T):
//   v_kt = alpha_k v_k,t-1 + beta_k (|eps_t-1| - c) + gamma_k eps_t-1   (v_k1 = v0_k)
//   s_t  = log sigma_Y + (1/2) sum_k v_kt          (= log h_t)
//   eps_t = (y_t - mu_Y) exp(-s_t)
//   l_t  = -(1/2) log 2pi - s_t + log sum_i exp(x_it),
//   x_it = log p_i + log a_i - (1/2) ((eps_t - mu_i) a_i)^2,   a_i = 1 / sigma_i.
// Reverse sweep (carry vb_k = dL/dv_k,t+1, zero after T):
//   r_i = softmax_i(x_it),  e_t = -sum_i r_i (eps_t - mu_i) a_i^2 + sum_k vb_k (beta_k sgn eps_t + gamma_k)
//   sb_t = -1 - e_t eps_t,  vb_k <- sb_t / 2 + alpha_k vb_k
//   d mu_Y -= e_t exp(-s_t);  d log sigma_Y += sb_t;
//   d alpha_k += vb_k v_k,t-1;  d beta_k += vb_k (|eps_t-1| - c);  d gamma_k += vb_k eps_t-1   (t >= 2)
//   d log p_i += r_i;  d mu_i += r_i (eps_t - mu_i) a_i^2;  d a_i += r_i (1/a_i - (eps_t - mu_i)^2 a_i)
// then through Table 1's transforms and (EGARCH_tran1)-(EGARCH_tran2); the
// mixture normalisation's Jacobian is taken by forward-mode duals.
// Memory: the state (v_k, eps) is checkpointed every kSeg observations in the
// forward pass; the reverse sweep recomputes one segment at a time into a
// per-thread shared-memory buffer.  Per-segment sums are in Real and added
// into FP64 accumulators every kFlushSegs segments.
#pragma once

#include "recursion.cuh"

namespace smc {

template <typename Real>
__device__ __forceinline__ Real nexp(Real x)
{
    if constexpr (sizeof(Real) == 4) return ex2_approx(x * (float)kLog2e);
    else return exp(x);
}

template <typename Real>
__device__ __forceinline__ Real nlog(Real x)
{
    if constexpr (sizeof(Real) == 4) return lg2_approx(x) * (float)kLn2;
    else return log(x);
}

template <typename Real>
struct Dual {
    Real v, d;
};
template <typename Real> __device__ __forceinline__ Dual<Real> dadd(Dual<Real> a, Dual<Real> b) { return {a.v + b.v, a.d + b.d}; }
template <typename Real> __device__ __forceinline__ Dual<Real> dsub(Dual<Real> a, Dual<Real> b) { return {a.v - b.v, a.d - b.d}; }
template <typename Real> __device__ __forceinline__ Dual<Real> dmul(Dual<Real> a, Dual<Real> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename Real> __device__ __forceinline__ Dual<Real> ddiv(Dual<Real> a, Dual<Real> b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }

// Mixture parameters (log p_i, mu_i, a_i = 1/sigma_i) from theta_6i, theta_7i,
// theta_8i with tangents along one input direction.
template <typename Real, int I>
__device__ void mixture_dual(const Real* th6, const Real* th7, const Real* th8, int dir,
                             Dual<Real>* logp, Dual<Real>* mu, Dual<Real>* a)
{
    Dual<Real> ps[I], ms[I], ss[I];
#pragma unroll
    for (int i = 0; i < I; ++i) {
        // p* = tanh(theta_6) + 1 = 2 / (1 + exp(-2 theta_6)), dp*/dtheta_6 = p* (2 - p*)
        const Real e = exp(Real(-2) * th6[i]);
        const Real p = Real(2) / (Real(1) + e);
        ps[i] = {p, dir == i ? p * (Real(2) - p) : Real(0)};
        ms[i] = {th7[i], dir == I + i ? Real(1) : Real(0)};
        const Real s = exp(th8[i]);
        ss[i] = {s, dir == 2 * I + i ? s : Real(0)};
    }
    Dual<Real> S = {Real(0), Real(0)};
#pragma unroll
    for (int i = 0; i < I; ++i) S = dadd(S, ps[i]);
    Dual<Real> pn[I], m = {Real(0), Real(0)};
#pragma unroll
    for (int i = 0; i < I; ++i) {
        pn[i] = ddiv(ps[i], S);
        m = dadd(m, dmul(pn[i], ms[i]));
    }
    Dual<Real> V = {Real(0), Real(0)}, m2[I];
#pragma unroll
    for (int i = 0; i < I; ++i) {
        m2[i] = dsub(ms[i], m);
        V = dadd(V, dmul(pn[i], dadd(dmul(m2[i], m2[i]), dmul(ss[i], ss[i]))));
    }
    const Real sq = sqrt(V.v);
    const Dual<Real> c = {Real(1) / sq, -V.d / (Real(2) * V.v * sq)};
#pragma unroll
    for (int i = 0; i < I; ++i) {
        logp[i] = {log(pn[i].v), pn[i].d / pn[i].v};
        mu[i] = dmul(c, m2[i]);
        const Dual<Real> sg = dmul(c, ss[i]);
        a[i] = {Real(1) / sg.v, -sg.d / (sg.v * sg.v)};
    }
}

// Natural-unit recursion with its adjoint.
template <typename Real, int K, int I>
struct EgarchNat {
    static constexpr int kNp = 2 + 3 * K + 3 * I;   // mu, lsy, alpha, beta, gamma, log p, mu_i, a_i
    Real mu, lsy;
    Real al[K], be[K], ga[K], v0[K];
    Real lpa[I], lp[I], mi[I], a[I];
    Real v[K], eps;
    int eps0_zero;

    __device__ __forceinline__ void setup(const Real* th, int has_gamma, int e0z)
    {
        EgarchParams<Real, K, I> q;
        egarch_transform<Real, K, I>(th, has_gamma, q);
        mu = q.mu_y;
        lsy = q.log_sigma_y;
        eps0_zero = e0z;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            al[k] = q.alpha[k];
            be[k] = q.beta[k];
            ga[k] = q.gamma[k];
            v0[k] = e0z ? -q.beta[k] * (Real)kSqrt2OverPi : Real(0);
        }
#pragma unroll
        for (int i = 0; i < I; ++i) {
            a[i] = Real(1) / q.sig[i];
            mi[i] = q.mu[i];
            lp[i] = log(q.p[i]);
            lpa[i] = lp[i] + log(a[i]);
        }
        eps = Real(0);
    }

    // One observation's state update only: (v, eps) and exp(-s_t).
    template <bool kFirst>
    __device__ __forceinline__ void step_state(Real y, Real& inv)
    {
        if constexpr (kFirst) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = v0[k];
        } else {
            const Real ae = fabs(eps) - (Real)kSqrt2OverPi;
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = al[k] * v[k] + be[k] * ae + ga[k] * eps;
        }
        Real vs = v[0];
#pragma unroll
        for (int k = 1; k < K; ++k) vs += v[k];
        inv = nexp<Real>(-(lsy + Real(0.5) * vs));
        eps = (y - mu) * inv;
    }

    // One observation: updates (v, eps), returns l_t + (1/2) log 2pi and exp(-s_t).
    template <bool kFirst>
    __device__ __forceinline__ Real step(Real y, Real& inv)
    {
        if constexpr (kFirst) {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = v0[k];
        } else {
            const Real ae = fabs(eps) - (Real)kSqrt2OverPi;
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = al[k] * v[k] + be[k] * ae + ga[k] * eps;
        }
        Real vs = v[0];
#pragma unroll
        for (int k = 1; k < K; ++k) vs += v[k];
        const Real s = lsy + Real(0.5) * vs;
        inv = nexp<Real>(-s);
        eps = (y - mu) * inv;
        if constexpr (I == 1) {
            return -s - Real(0.5) * eps * eps;
        } else {
            Real x[I], m = -INFINITY;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const Real z = (eps - mi[i]) * a[i];
                x[i] = lpa[i] - Real(0.5) * z * z;
                m = fmax(m, x[i]);
            }
            Real sum = 0;
#pragma unroll
            for (int i = 0; i < I; ++i) sum += nexp<Real>(x[i] - m);
            return -s + m + nlog<Real>(sum);
        }
    }
};

// Gradient of the natural parameters -> gradient with respect to the full
// theta vector (Table 1 layout).
template <typename Real, int K, int I>
__device__ void natural_to_theta(const EgarchNat<Real, K, I>& m, const double* gn, const Real* th,
                                 int has_gamma, double* gth)
{
    int j = 0;
    gth[j++] = gn[0] / 1000.0;
    gth[j++] = gn[1];
#pragma unroll
    for (int k = 0; k < K; ++k) gth[j++] = gn[2 + k] * (1.0 - (double)m.al[k] * (double)m.al[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) gth[j++] = gn[2 + K + k] * (double)m.be[k];
    if (has_gamma) {
#pragma unroll
        for (int k = 0; k < K; ++k) gth[j++] = gn[2 + 2 * K + k];
    }
    if constexpr (I >= 2) {
        const Real* th6 = th + j;
        for (int dir = 0; dir < 3 * I; ++dir) {
            Dual<Real> lpd[I], mud[I], ad[I];
            mixture_dual<Real, I>(th6, th6 + I, th6 + 2 * I, dir, lpd, mud, ad);
            double g = 0.0;
#pragma unroll
            for (int i = 0; i < I; ++i)
                g += gn[2 + 3 * K + i] * (double)lpd[i].d + gn[2 + 3 * K + I + i] * (double)mud[i].d +
                     gn[2 + 3 * K + 2 * I + i] * (double)ad[i].d;
            gth[j + dir] = g;
        }
    }
}

// Forward pass from t = 1 to T with checkpoints every kSeg observations:
// ckpt[seg][k][P] holds (v_1..v_K, eps) after observation seg*kSeg (1-based)
// is processed, for seg = 0.. (the state entering segment seg + 1).
// Returns l(theta); leaves the end state in m.
template <typename Real, int K, int I, int kSeg>
__device__ double adj_forward(EgarchNat<Real, K, I>& m, const Real* __restrict__ y, int T, Real* ckpt,
                              size_t P, int p, bool write)
{
    double acc = 0.0;
    Real part = 0;
    const int nseg = (T + kSeg - 1) / kSeg;
    for (int sg = 0; sg < nseg; ++sg) {
        const int t0 = sg * kSeg, n = min(kSeg, T - t0);
        if (write && sg > 0) {
            Real* c = ckpt + (size_t)(sg - 1) * (K + 1) * P + p;
#pragma unroll
            for (int k = 0; k < K; ++k) c[k * P] = m.v[k];
            c[K * P] = m.eps;
        }
        for (int r = 0; r < n; ++r) {
            Real inv;
            const Real yy = y[t0 + r];
            part += (t0 + r == 0) ? m.template step<true>(yy, inv) : m.template step<false>(yy, inv);
        }
        if ((sg & 7) == 7 || sg == nseg - 1) {
            acc += (double)part;
            part = 0;
        }
    }
    return acc + (double)T * (-0.5 * kLog2Pi);
}

// FP32 forward pass through the base-2 recursion of the random-walk kernel
// (EgarchF32), writing the same natural-unit checkpoints as adj_forward.
template <int K, int I, int kSeg>
__device__ double adj_forward_fast(const float* th, int has_gamma, int eps0_zero, const float* __restrict__ y,
                                   int T, float* ckpt, size_t P, int p)
{
    static_assert(32 % kSeg == 0, "FP32 partials of 32 observations cover whole segments");
    constexpr int kPerPartial = 32 / kSeg;
    EgarchF32<K, I> f;
    f.setup(th, has_gamma, eps0_zero);
    const int nseg = (T + kSeg - 1) / kSeg;
    for (int sg = 0; sg < nseg; ++sg) {
        const int t0 = sg * kSeg, n = min(kSeg, T - t0);
        if (sg > 0) {
            // the state in natural units, converted in FP32 (it is stored in
            // FP32): v_k = 2 ln2 v'_k (v'_1 less log2 sigma_Y - log2 s), eps = es / s
            float* c = ckpt + (size_t)(sg - 1) * (K + 1) * P + p;
#pragma unroll
            for (int k = 0; k < K; ++k) c[k * P] = (k == 0 ? f.v[0] - f.lsy2p : f.v[k]) * (float)(2.0 * kLn2);
            c[K * P] = f.es * (float)(1.0 / kSfac);
        }
        if (n == kSeg && t0 > 0) {
#pragma unroll 8
            for (int r = 0; r < kSeg; ++r) f.template step<false>(y[t0 + r]);
        } else {
            for (int r = 0; r < n; ++r) {
                if (t0 + r == 0) f.template step<true>(y[0]);
                else f.template step<false>(y[t0 + r]);
            }
        }
        if (sg % kPerPartial == kPerPartial - 1 || sg == nseg - 1) {
            f.flush();
            if (sg % (8 * kPerPartial) == 8 * kPerPartial - 1) f.flush_fp64();
        }
    }
    return f.finish(T);
}

// Reverse sweep over all segments; gn (double, kNp) receives d l / d natural
// parameters.  buf is this thread's shared-memory slab laid out
// [kSeg][K + 2][stride] (v_k, eps, exp(-s)) with element (t, f) at
// buf[(t * (K + 2) + f) * stride].
template <typename Real, int K, int I, int kSeg>
__device__ void adj_reverse(EgarchNat<Real, K, I> m, const Real* __restrict__ y, int T, const Real* ckpt,
                            size_t P, int p, Real* buf, int stride, double* gn)
{
    constexpr int NP = EgarchNat<Real, K, I>::kNp;
    constexpr int W = K + 2;
    Real gs[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) gs[i] = 0;
    for (int i = 0; i < NP; ++i) gn[i] = 0.0;
    Real vb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vb[k] = 0;
    const Real c0 = (Real)kSqrt2OverPi;
    // per-particle constants of the step below
    Real a2[I], sgi[I], bp[K], bm[K];
#pragma unroll
    for (int i = 0; i < I; ++i) {
        a2[i] = m.a[i] * m.a[i];
        sgi[i] = Real(1) / m.a[i];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        bp[k] = m.be[k] + m.ga[k];   // beta sgn(eps) + gamma for eps > 0
        bm[k] = m.ga[k] - m.be[k];   // and for eps < 0
    }
    // One reverse step at observation t: state (eps_t, exp(-s_t)), previous
    // state (v_k,t-1, eps_t-1); has_prev: t >= 1 (0-based), i.e. v_k,t came
    // from the recursion rather than from v_k0.
    auto back = [&](Real eps, Real inv, const Real* vp, Real ep, bool has_prev) {
        Real dle;
        if constexpr (I == 1) {
            dle = -eps;
        } else {
            Real x[I], dz[I], mx = -INFINITY;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                dz[i] = eps - m.mi[i];
                const Real z = dz[i] * m.a[i];
                x[i] = m.lpa[i] - Real(0.5) * z * z;
                mx = fmax(mx, x[i]);
            }
            Real sum = 0;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                x[i] = nexp<Real>(x[i] - mx);
                sum += x[i];
            }
            Real isum;
            if constexpr (sizeof(Real) == 4) isum = __fdividef(1.0f, sum);   // sum in [1, I]
            else isum = Real(1) / sum;
            dle = 0;
#pragma unroll
            for (int i = 0; i < I; ++i) {
                const Real ri = x[i] * isum;
                const Real t = ri * dz[i] * a2[i];
                dle -= t;
                gs[2 + 3 * K + i] += ri;
                gs[2 + 3 * K + I + i] += t;
                gs[2 + 3 * K + 2 * I + i] += ri * (sgi[i] - dz[i] * dz[i] * m.a[i]);
            }
        }
        Real eb = dle;
#pragma unroll
        for (int k = 0; k < K; ++k) eb += vb[k] * (eps > Real(0) ? bp[k] : (eps < Real(0) ? bm[k] : m.ga[k]));
        const Real sb = Real(-1) - eb * eps;
        gs[0] -= eb * inv;
        gs[1] += sb;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            vb[k] = Real(0.5) * sb + m.al[k] * vb[k];
            if (has_prev) {
                gs[2 + k] += vb[k] * vp[k];
                gs[2 + K + k] += vb[k] * (fabs(ep) - c0);
                gs[2 + 2 * K + k] += vb[k] * ep;
            } else if (m.eps0_zero) {
                gs[2 + K + k] += vb[k] * (-c0);
            }
        }
    };
    const int nseg = (T + kSeg - 1) / kSeg;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int t0 = sg * kSeg, n = min(kSeg, T - t0);
        // state entering the segment
        Real vprev[K], eprev = 0;
        if (sg > 0) {
            const Real* c = ckpt + (size_t)(sg - 1) * (K + 1) * P + p;
#pragma unroll
            for (int k = 0; k < K; ++k) vprev[k] = c[k * P];
            eprev = c[K * P];
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) vprev[k] = 0;
        }
        // recompute the segment
#pragma unroll
        for (int k = 0; k < K; ++k) m.v[k] = vprev[k];
        m.eps = eprev;
        auto put = [&](int r, Real inv) {
#pragma unroll
            for (int k = 0; k < K; ++k) buf[(r * W + k) * stride] = m.v[k];
            buf[(r * W + K) * stride] = m.eps;
            buf[(r * W + K + 1) * stride] = inv;
        };
        if (n == kSeg && t0 > 0) {
#pragma unroll 8
            for (int r = 0; r < kSeg; ++r) {
                Real inv;
                m.template step_state<false>(y[t0 + r], inv);
                put(r, inv);
            }
        } else {
            for (int r = 0; r < n; ++r) {
                Real inv;
                if (t0 + r == 0) m.template step_state<true>(y[0], inv);
                else m.template step_state<false>(y[t0 + r], inv);
                put(r, inv);
            }
        }
        // reverse through the segment: observations t0 + n - 1 .. t0 + 1 take
        // their previous state from the buffer, observation t0 from the
        // checkpoint; only the first observation of the series (t = 0) has no
        // previous shock
        const Real* q = buf + (size_t)(n - 1) * W * stride;
        // unrolled by two: a step's mixture terms (independent of the adjoint
        // carry vb) overlap the previous step's carry update (measured on
        // K=2, I=2, T=5000, 262,144 particles: 5.90 ms per MALA launch against
        // 6.39 ms unrolled once, 5.96 ms by four)
#pragma unroll 2
        for (int r = n - 1; r >= 1; --r, q -= W * stride) {
            const Real* qp = q - W * stride;
            Real vp[K];
#pragma unroll
            for (int k = 0; k < K; ++k) vp[k] = qp[k * stride];
            back(q[K * stride], q[(K + 1) * stride], vp, qp[K * stride], true);
        }
        back(buf[K * stride], buf[(K + 1) * stride], vprev, eprev, t0 > 0);
        if ((sg & 7) == 0 || sg == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                gn[i] += (double)gs[i];
                gs[i] = 0;
            }
        }
    }
    for (int i = 0; i < NP; ++i) gn[i] += (double)gs[i];
}

}  // namespace smc
