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
