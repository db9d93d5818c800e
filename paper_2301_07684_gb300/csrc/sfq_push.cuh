// sfq_push.cuh -- the Boris push of the momenta, the particle pusher a PIC code runs between
// Monte Carlo steps (Boris 1970).  The paper's library leaves the push to the host code; it
// is here so that the step can be coupled to moving particles in the same field sources.
//
// Normalised units of the step: du/dt = q (E + u x B / gamma), u = p / m c, q in units of |e|
// (electron -1, positron +1, photon 0: photons move freely), fields in E_r, time in 1/omega_r.
//   u- = u + q E dt/2;  t = q B dt / (2 gamma(u-));  s = 2 t / (1 + t.t);
//   u' = u- + u- x t;  u+ = u- + u' x s;  u_new = u+ + q E dt/2.
#pragma once
#include "sfq_step.cuh"

namespace sfq {

template <typename T>
__device__ __forceinline__ void boris(T u[3], const T E[3], const T B[3], T q, T dt) {
    const T h = (T)0.5 * q * dt;
    T um[3], t[3], s[3], up[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = fma(h, E[k], u[k]);
    const T gm = sqrt(fma(um[0], um[0], fma(um[1], um[1], fma(um[2], um[2], (T)1))));
    const T hg = h / gm;
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = hg * B[k];
    const T f = (T)2 / fma(t[0], t[0], fma(t[1], t[1], fma(t[2], t[2], (T)1)));
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = f * t[k];
    const T c0 = um[1] * t[2] - um[2] * t[1], c1 = um[2] * t[0] - um[0] * t[2], c2 = um[0] * t[1] - um[1] * t[0];
    const T v0 = um[0] + c0, v1 = um[1] + c1, v2 = um[2] + c2;
    up[0] = um[0] + (v1 * s[2] - v2 * s[1]);
    up[1] = um[1] + (v2 * s[0] - v0 * s[2]);
    up[2] = um[2] + (v0 * s[1] - v1 * s[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = fma(h, E[k], up[k]);
}

// One push of every alive lepton of the population at the launch's step (fields as the
// step reads them); photons and dead particles are left as they are.
template <typename T, int FK>
__global__ void __launch_bounds__(256) push_kernel(const StepArgs<T> a, T dt) {
    const int64_t n = effective_n(a);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t fl = a.flags[i];
        const int sp = (fl >> SFQ_SPECIES_SHIFT) & 3;
        if (!(fl & SFQ_ALIVE) || sp == SFQ_PHOTON) continue;
        T E[3], B[3];
        load_fields<T, FK>(a, i, E, B);
        T u[3] = {a.px[i], a.py[i], a.pz[i]};
        boris<T>(u, E, B, sp == SFQ_ELECTRON ? (T)-1 : (T)1, dt);
        a.px[i] = u[0]; a.py[i] = u[1]; a.pz[i] = u[2];
    }
}

}  // namespace sfq
