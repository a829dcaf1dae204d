// Reverse-mode entry points (force VJP, density loss, step factors) and the energies with the
// Layzer-Irvine bookkeeping.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <vector>

#include "host_internal.h"

using namespace p3m_host;

// ---------------------------------------------------------------- reverse-mode derivatives

extern "C" int p3m_step_factors(const p3m_ctx *c, double a, double da, double *k1, double *dfac,
                                double *k2)
{
    if (!c || !finite_pos(a) || !finite_pos(da)) return P3M_EINVAL;
    const double am = a + 0.5 * da, a2 = a + da;
    if (k1) *k1 = c->mass * p3m_kick_factor(c->cosmo, a, am);
    if (dfac) *dfac = p3m_drift_factor(c->cosmo, a, a2) / c->mass;
    if (k2) *k2 = c->mass * p3m_kick_factor(c->cosmo, am, a2);
    return P3M_OK;
}

extern "C" int p3m_axpy(p3m_ctx *c, double alpha, const double *x3n, double *y3n)
{
    if (!c || !x3n || !y3n) return fail(c, P3M_EINVAL, "p3m_axpy: NULL argument");
    CK(launch_axpy(c, y3n, x3n, alpha));
    return P3M_OK;
}

extern "C" int p3m_force_vjp(p3m_ctx *c, const double *v3n, double *out3n, int on_device)
{
    if (!c || !v3n || !out3n) return fail(c, P3M_EINVAL, "p3m_force_vjp: NULL argument");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_force_vjp: no particles loaded");
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    // sort, cells and mesh fields at the current positions (the pair forces are not needed)
    int rc = key_current(c);
    if (!rc) rc = evaluate(c, 0.0, nullptr, false, false);
    if (rc) return rc;
    c->forces_valid = !c->short_range;
    const double *vin = v3n;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->pos_alt, v3n, bytes, cudaMemcpyHostToDevice, c->stream));
        vin = c->pos_alt;
    }
    CK(launch_to_slots(c, vin, c->adj_vs));
    CK(launch_force_vjp(c, c->adj_vs, c->adj_out));
    if (on_device) {
        CK(launch_scatter_out(c, c->adj_out, out3n));
        return P3M_OK;
    }
    CK(launch_scatter_out(c, c->adj_out, c->pos_alt));
    CK(cudaMemcpyAsync(out3n, c->pos_alt, bytes, cudaMemcpyDeviceToHost, c->stream));
    return check_flags(c);
}

extern "C" int p3m_density_loss(p3m_ctx *c, const double *target, double *loss, double *grad3n,
                                int on_device)
{
    if (!c || !target || !loss) return fail(c, P3M_EINVAL, "p3m_density_loss: NULL argument");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_density_loss: no particles loaded");
    const size_t M3 = (size_t)c->g.mesh * c->g.mesh * c->g.mesh;
    const size_t bytes = 3 * sizeof(double) * (size_t)c->g.n;
    const double *t = target;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->adj_u, target, sizeof(double) * M3, cudaMemcpyHostToDevice, c->stream));
        t = (const double *)c->adj_u;
    }
    CK(launch_deposit(c));
    double *loss_dev = c->red + 1024 * 4 + 4;
    CK(launch_density_loss(c, t, loss_dev, grad3n ? c->adj_out : nullptr));
    if (grad3n) {
        if (on_device) {
            CK(launch_scatter_out(c, c->adj_out, grad3n));
        } else {
            CK(launch_scatter_out(c, c->adj_out, c->pos_alt));
            CK(cudaMemcpyAsync(grad3n, c->pos_alt, bytes, cudaMemcpyDeviceToHost, c->stream));
        }
    }
    CK(cudaMemcpyAsync(loss, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return P3M_OK;
}

// ---------------------------------------------------------------- energies

namespace {

// phi_per - phi_iso: the long-range potential a particle feels from its own periodic images
// (with the neutralising background), by the Ewald identity at alpha = 2.6/L for the lattice
// sum and the split's alpha = 1/(2 r_s) for the short-range images:
//   (4 pi/L^3) sum_{k != 0} exp(-k^2 r_s^2)/k^2 = psi_self - sum_{n != 0} erfc(|n|L/(2 r_s))/(|n|L)
//                                                  + 4 pi r_s^2/L^3 + 1/(sqrt(pi) r_s),
// psi_self the alpha-independent Ewald self term of one particle per cell.
double image_potential(const P3MGeom &g)
{
    const double L = g.box, alpha = 2.6 / L, rs = g.r_s;
    double real = 0.0, recip = 0.0, srimg = 0.0;
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) {
                if (!x && !y && !z) continue;
                const double r = L * sqrt((double)(x * x + y * y + z * z));
                real += erfc(alpha * r) / r;
                srimg += erfc(0.5 * r / rs) / r;
            }
    const double kf = 2.0 * M_PI / L;
    for (int x = -8; x <= 8; ++x)
        for (int y = -8; y <= 8; ++y)
            for (int z = -8; z <= 8; ++z) {
                if (!x && !y && !z) continue;
                const double k2 = kf * kf * (double)(x * x + y * y + z * z);
                recip += exp(-k2 / (4.0 * alpha * alpha)) / k2;
            }
    const double V = L * L * L;
    const double psi_self = real + 4.0 * M_PI / V * recip - M_PI / (alpha * alpha * V) -
                            2.0 * alpha / sqrt(M_PI);
    const double ksum = psi_self - srimg + 4.0 * M_PI * rs * rs / V + 1.0 / (sqrt(M_PI) * rs);
    return -g.gm * ksum + g.gm / (sqrt(M_PI) * rs);  // phi_per - phi_iso
}

}  // namespace

namespace p3m_host {

int energy_now(p3m_ctx *c, double *kin, double *pot)
{
    int rc = key_current(c);
    if (!rc) rc = evaluate(c, 0.0, nullptr, false, false);
    if (rc) return rc;
    double cst = 0.0;
    if (c->short_range) {
        const double V = c->g.box * c->g.box * c->g.box;
        cst = image_potential(c->g) + 4.0 * M_PI * c->g.gm * ((double)c->g.n / V) * c->g.r_s * c->g.r_s;
    }
    double *sum_dev = c->red + 1024 * 4 + 5;
    CK(launch_potential(c, cst, c->adj_out, sum_dev));
    double sum = 0.0, r[4];
    CK(cudaMemcpyAsync(&sum, sum_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(launch_diag(c, r));  // synchronises
    *pot = 0.5 * c->mass * sum / c->a;
    *kin = r[3] / (2.0 * c->mass * c->a * c->a);
    c->forces_valid = !c->short_range;
    return P3M_OK;
}

}  // namespace p3m_host

extern "C" int p3m_energy(p3m_ctx *c, double *kinetic, double *potential)
{
    if (!c || !kinetic || !potential) return fail(c, P3M_EINVAL, "p3m_energy: NULL argument");
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_energy: no particles loaded");
    return energy_now(c, kinetic, potential);
}

extern "C" int p3m_track_energy(p3m_ctx *c, int enable)
{
    if (!c) return P3M_EINVAL;
    if (!enable) {
        if (c->track_energy) ++c->geom_version;
        c->track_energy = false;
        return P3M_OK;
    }
    if (!c->have_particles) return fail(c, P3M_ESTATE, "p3m_track_energy: no particles loaded");
    double k0 = 0.0, w0 = 0.0;
    int rc = energy_now(c, &k0, &w0);
    if (rc) return rc;
    double p2 = 2.0 * c->mass * c->a * c->a * k0;
    const double li0[4] = {0.0, p2, c->a, 0.0};
    CK(cudaMemcpyAsync(c->li, li0, sizeof(li0), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->li_a0 = c->a;
    c->li_e0 = c->a * (k0 + w0);
    c->track_energy = true;
    ++c->geom_version;  // captured steps lack the tracking kernels
    return P3M_OK;
}

