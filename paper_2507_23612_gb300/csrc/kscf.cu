// Fixed-V_eff DFT+U SCF with Brillouin-zone sampling over one handle per k-point.
//
// Eq. (orbital_occup_ext) averages the occupation matrices over the Brillouin zone:
// D = sum_k w_k D_k (weights summing to one).  One Fermi level spans every (spin, k)
// channel, every k-point's Hamiltonian carries the same D, and D is Pulay-mixed every
// iteration (Sec. II.B).  D is complex Hermitian in general; its real and imaginary parts
// are mixed as one real vector.  A real (Gamma-point) handle needs a real D: a k-set that
// holds it must be closed under k -> -k (D_-k = conj D_k keeps D real).
//
// Every grid-sized step runs in the handles' kernels (Lanczos bounds, Chebyshev filter,
// Rayleigh-Ritz, occupation matrices); this file holds the driver's scalar host work:
// the Fermi level over the k-weighted states, the energy sums over the 25 numbers per
// Hubbard atom and channel, and Pulay on them.
#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "hub_internal.cuh"

struct hub_kscf {
    int nk = 0;
    std::vector<hub_t> hubs;
    std::vector<double> kw;
    hub_scf_params p{};
    int nhub = 0;
    std::vector<double> U;                         // per Hubbard atom (Ha)
    std::vector<void*> X;                          // [nspin * nk], index s * nk + k
    std::vector<const void*> v0;
    std::vector<double> Dr_in, Di_in, Dr_out, Di_out;  // [nspin * nhub * 25]
    std::vector<double> eig, occ;                  // [nspin * nk * ncol]
    std::vector<std::array<double, 3>> bounds;     // a_low, a, b per channel
    std::vector<char> have_bounds;
    std::vector<std::vector<double>> hx, hr;       // Pulay history of [Re D, Im D]
    int iter = 0, small = 0;
    bool have_prev = false;
    double E_prev = 0.0;
    hub_scf_result last{};
    std::string err;
};

namespace {

int kfail(hub_kscf_t s, int code, const std::string& msg) {
    if (s) s->err = msg;
    return code;
}

// a handle call's status, with that handle's message carried over
int kcall(hub_kscf_t s, hub_t h, int rc, const char* what) {
    if (rc == HUB_OK) return rc;
    const char* m = hub_last_error(h);
    return kfail(s, rc, std::string(what) + ": " + (m ? m : ""));
}

}  // namespace

extern "C" {

int hub_kscf_create(hub_kscf_t* out, int nk, hub_t const* hubs, const double* kweights,
                    const hub_scf_params* p, void* const* X, const void* const* v0,
                    const double* D0_re, const double* D0_im) {
    if (!out) return HUB_EINVAL;
    *out = nullptr;
    if (nk < 1 || !hubs || !kweights || !p || !X || !v0) return HUB_EINVAL;
    if (p->nspin < 1 || p->nspin > 2 || p->ncol < 1 || p->degree < 1 || p->max_iter < 1 ||
        p->lanczos_steps < 1 || p->lanczos_steps > 64 || p->density)
        return HUB_EINVAL;
    double wsum = 0.0;
    for (int k = 0; k < nk; ++k) {
        if (!hubs[k] || !(kweights[k] >= 0.0)) return HUB_EINVAL;
        wsum += kweights[k];
    }
    if (std::fabs(wsum - 1.0) > 1e-12) return HUB_EINVAL;
    const hub_t h0 = hubs[0];
    for (int k = 0; k < nk; ++k) {
        const hub_t h = hubs[k];
        if (h->Nd != h0->Nd || h->prec != h0->prec || !h->atoms_set || !h->veff_set ||
            h->proj.nhub != h0->proj.nhub || (long)p->ld < h->Nd)
            return HUB_EINVAL;
    }
    const int ns = p->nspin, nh = h0->proj.nhub;
    for (int q = 0; q < ns * nk; ++q)
        if (!X[q] || !v0[q]) return HUB_EINVAL;
    if (nh > 0 && !D0_re) return HUB_EINVAL;
    auto* s = new hub_kscf();
    s->nk = nk;
    s->hubs.assign(hubs, hubs + nk);
    s->kw.assign(kweights, kweights + nk);
    s->p = *p;
    s->nhub = nh;
    s->U = h0->proj.h_U;
    s->X.assign(X, X + (size_t)ns * nk);
    s->v0.assign(v0, v0 + (size_t)ns * nk);
    const size_t nD = (size_t)ns * nh * 25;
    s->Dr_in.assign(nD, 0.0);
    s->Di_in.assign(nD, 0.0);
    if (D0_re) std::copy(D0_re, D0_re + nD, s->Dr_in.begin());
    if (D0_im) std::copy(D0_im, D0_im + nD, s->Di_in.begin());
    s->Dr_out.assign(nD, 0.0);
    s->Di_out.assign(nD, 0.0);
    s->eig.assign((size_t)ns * nk * p->ncol, 0.0);
    s->occ.assign(s->eig.size(), 0.0);
    s->bounds.assign((size_t)ns * nk, {0.0, 0.0, 0.0});
    s->have_bounds.assign((size_t)ns * nk, 0);
    *out = s;
    return HUB_OK;
}

int hub_kscf_destroy(hub_kscf_t s) {
    delete s;
    return HUB_OK;
}

const char* hub_kscf_last_error(hub_kscf_t s) { return s ? s->err.c_str() : "NULL k-point SCF"; }

}  // extern "C"

namespace {

// phase 1: D_in into every handle (a real handle takes a real D only)
int kscf_set_D(hub_kscf_t s) {
    const int ns = s->p.nspin;
    const size_t per = (size_t)s->nhub * 25;
    double imax = 0.0;
    for (double v : s->Di_in) imax = std::max(imax, std::fabs(v));
    int rc;
    for (int k = 0; k < s->nk; ++k) {
        const hub_t h = s->hubs[k];
        if (!h->cplx && imax > 1e-10)
            return kfail(s, HUB_EINVAL, "a real (Gamma) k-point needs a real D: use a k-set closed under k -> -k");
        for (int sp = 0; sp < ns; ++sp)
            if ((rc = kcall(s, h, hub_set_occupation_matrix(h, sp, s->Dr_in.data() + sp * per,
                                                           h->cplx ? s->Di_in.data() + sp * per : nullptr),
                            "hub_set_occupation_matrix")))
                return rc;
    }
    return HUB_OK;
}

int kscf_passes(hub_kscf_t s) { return s->iter == 0 ? std::max(1, s->p.first_passes) : 1; }

// filter bounds of channel c (spin c / nk, k-point c % nk): Lanczos the first time
int kscf_bounds(hub_kscf_t s, int c) {
    if (s->have_bounds[c]) return HUB_OK;
    const hub_t h = s->hubs[c % s->nk];
    double lo, up;
    int rc;
    if ((rc = kcall(s, h, hub_lanczos_bound(h, c / s->nk, s->p.lanczos_steps, s->v0[c], &lo, &up), "hub_lanczos_bound")))
        return rc;
    s->bounds[c] = {lo, lo + 0.1 * (up - lo), up};
    s->have_bounds[c] = 1;
    return HUB_OK;
}

// Rayleigh-Ritz of channel c; the next filter's a_low and a from its Ritz values
int kscf_rr(hub_kscf_t s, int c) {
    const hub_t h = s->hubs[c % s->nk];
    const int n = s->p.ncol;
    double* eg = s->eig.data() + (size_t)c * n;
    int rc;
    if ((rc = kcall(s, h, hub_rayleigh_ritz(h, c / s->nk, s->X[c], n, s->p.ld, eg, nullptr), "hub_rayleigh_ritz")))
        return rc;
    s->bounds[c][0] = eg[0];
    s->bounds[c][1] = eg[n - 1];
    return HUB_OK;
}

// Rayleigh-Ritz of the two spin channels of k-point k (one handle): both subspace
// eigenproblems in one launch
int kscf_rr_pair(hub_kscf_t s, int k) {
    const hub_t h = s->hubs[k];
    const int n = s->p.ncol, c0 = k, c1 = s->nk + k;
    void* X[2] = {s->X[c0], s->X[c1]};
    double* eg[2] = {s->eig.data() + (size_t)c0 * n, s->eig.data() + (size_t)c1 * n};
    int rc;
    if ((rc = kcall(s, h, hub::rr_two_spins(h, X, n, s->p.ld, eg), "Rayleigh-Ritz of both spins"))) return rc;
    for (int c : {c0, c1}) {
        s->bounds[c][0] = s->eig[(size_t)c * n];
        s->bounds[c][1] = s->eig[(size_t)c * n + n - 1];
    }
    return HUB_OK;
}

// phase 3: Fermi level, D_out, energy, convergence and Pulay mixing of D
int kscf_post(hub_kscf_t s, hub_scf_result* res) {
    const hub_scf_params& p = s->p;
    const int ns = p.nspin, nk = s->nk, nh = s->nhub, n = p.ncol;
    const double deg = ns == 1 ? 2.0 : 1.0;
    const size_t per = (size_t)nh * 25;
    int rc;
    // one Fermi level over every (spin, k) state, each weighted by its k-point's weight
    const int nstates = ns * nk * n;
    std::vector<double> w((size_t)nstates);
    for (int c = 0; c < ns * nk; ++c) std::fill(w.begin() + (size_t)c * n, w.begin() + (size_t)(c + 1) * n, s->kw[c % nk]);
    double mu = 0.0;
    if ((rc = hub_fermi_dirac(nstates, s->eig.data(), w.data(), p.kT, p.n_elec, deg, s->occ.data(), &mu)))
        return kfail(s, rc, "hub_fermi_dirac: electron count outside the states' capacity");
    // D_out = sum_k w_k D_k (Eq. orbital_occup_ext)
    std::fill(s->Dr_out.begin(), s->Dr_out.end(), 0.0);
    std::fill(s->Di_out.begin(), s->Di_out.end(), 0.0);
    std::vector<double> dr(per), di(per);
    for (int sp = 0; sp < ns; ++sp)
        for (int k = 0; k < nk; ++k) {
            const hub_t h = s->hubs[k];
            const int c = sp * nk + k;
            if (nh == 0) continue;
            if ((rc = kcall(s, h, hub_occupation(h, sp, s->X[c], n, p.ld, s->occ.data() + (size_t)c * n, s->kw[k],
                                                 dr.data(), di.data(), nullptr), "hub_occupation")))
                return rc;
            for (size_t q = 0; q < per; ++q) {
                s->Dr_out[sp * per + q] += dr[q];
                s->Di_out[sp * per + q] += di[q];
            }
        }
    // energy: E = sum w f eig - sum_I Re sum_ab M_in,ab D_out,ba + E_U(D_out) - kT S
    double e_band = 0.0, e_dc = 0.0, e_u = 0.0, ent = 0.0;
    for (int i = 0; i < nstates; ++i) e_band += deg * w[i] * s->occ[i] * s->eig[i];
    for (int sp = 0; sp < ns; ++sp)
        for (int I = 0; I < nh; ++I) {
            const size_t o = sp * per + (size_t)I * 25;
            const double Uh = s->U[I];
            double dc = 0.0, tr = 0.0, tr2 = 0.0;
            for (int a = 0; a < 5; ++a) {
                tr += s->Dr_out[o + a * 5 + a];
                for (int b = 0; b < 5; ++b) {
                    const double Mr = 0.5 * Uh * ((a == b ? 1.0 : 0.0) - 2.0 * s->Dr_in[o + a * 5 + b]);
                    const double Mi = -Uh * s->Di_in[o + a * 5 + b];
                    const double Dbr = s->Dr_out[o + b * 5 + a], Dbi = s->Di_out[o + b * 5 + a];
                    dc += Mr * Dbr - Mi * Dbi;
                    tr2 += s->Dr_out[o + a * 5 + b] * Dbr - s->Di_out[o + a * 5 + b] * Dbi;
                }
            }
            e_dc += deg * dc;
            e_u += deg * 0.5 * Uh * (tr - tr2);
        }
    if (p.kT > 0)
        for (int c = 0; c < ns * nk; ++c) {
            std::vector<double> f(s->occ.begin() + (size_t)c * n, s->occ.begin() + (size_t)(c + 1) * n);
            ent += deg * s->kw[c % nk] * hub::fd_entropy(f);
        }
    const double E = e_band - e_dc + e_u - p.kT * ent;
    double dD = 0.0;
    for (size_t q = 0; q < s->Dr_in.size(); ++q)
        dD = std::max(dD, std::hypot(s->Dr_out[q] - s->Dr_in[q], s->Di_out[q] - s->Di_in[q]));
    const double dE = s->have_prev ? E - s->E_prev : 0.0;
    if (s->have_prev && std::fabs(dE) / std::max(1, p.natoms) < p.tol_e_atom) s->small++;
    else s->small = 0;
    s->have_prev = true;
    s->E_prev = E;
    s->iter++;
    hub_scf_result r{};
    r.iter = s->iter;
    r.converged = (s->small >= 2 && dD < p.tol_D) ? 1 : 0;
    r.E = E; r.E_band = e_band; r.E_U = e_u; r.dE = dE; r.dD = dD; r.mu = mu;
    for (int k = 0; k < nk; ++k) r.jacobi_sweeps = std::max(r.jacobi_sweeps, s->hubs[k]->last_sweeps);
    if (!r.converged) {
        // Pulay / DIIS on x = [Re D, Im D] with history p.pulay_history and mixing p.pulay_beta
        const size_t nD = s->Dr_in.size();
        std::vector<double> xin(2 * nD), rr(2 * nD);
        for (size_t q = 0; q < nD; ++q) {
            xin[q] = s->Dr_in[q];
            xin[nD + q] = s->Di_in[q];
            rr[q] = s->Dr_out[q] - s->Dr_in[q];
            rr[nD + q] = s->Di_out[q] - s->Di_in[q];
        }
        s->hx.push_back(xin);
        s->hr.push_back(rr);
        const int hist = std::max(1, p.pulay_history);
        while ((int)s->hx.size() > hist) { s->hx.erase(s->hx.begin()); s->hr.erase(s->hr.begin()); }
        const int k = (int)s->hr.size();
        std::vector<double> G((size_t)k * k, 0.0), coef;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                double sm = 0.0;
                for (size_t q = 0; q < 2 * nD; ++q) sm += s->hr[i][q] * s->hr[j][q];
                G[(size_t)i * k + j] = sm;
            }
        if (!hub::pulay_solve(G, k, coef)) { coef.assign(k, 0.0); coef[k - 1] = 1.0; }   // linear mixing
        for (size_t q = 0; q < 2 * nD; ++q) {
            double xs = 0.0, rs = 0.0;
            for (int i = 0; i < k; ++i) { xs += coef[i] * s->hx[i][q]; rs += coef[i] * s->hr[i][q]; }
            const double v = xs + p.pulay_beta * rs;
            if (q < nD) s->Dr_in[q] = v; else s->Di_in[q - nD] = v;
        }
    }
    s->last = r;
    if (res) *res = r;
    return HUB_OK;
}

}  // namespace

extern "C" {

int hub_kscf_iterate(hub_kscf_t s, hub_scf_result* res) {
    hub::NvtxRange nvtx_("hub_kscf_iterate");
    if (!s) return HUB_EINVAL;
    const hub_scf_params& p = s->p;
    int rc;
    if ((rc = kscf_set_D(s))) return rc;
    const int passes = kscf_passes(s);
    auto filter = [&](int c) {
        const hub_t h = s->hubs[c % s->nk];
        int r;
        if ((r = kscf_bounds(s, c))) return r;
        const auto& bd = s->bounds[c];
        return kcall(s, h, hub_chefsi_filter(h, c / s->nk, s->X[c], p.ncol, p.ld, p.degree, bd[1], bd[2], bd[0],
                                             nullptr), "hub_chefsi_filter");
    };
    if (p.nspin == 2) {
        // per k-point both spin channels, their Rayleigh-Ritz in one eigensolver launch
        for (int k = 0; k < s->nk; ++k)
            for (int pass = 0; pass < passes; ++pass) {
                if ((rc = filter(k)) || (rc = filter(s->nk + k))) return rc;
                if ((rc = kscf_rr_pair(s, k))) return rc;
            }
    } else {
        for (int c = 0; c < s->nk; ++c)
            for (int pass = 0; pass < passes; ++pass) {
                if ((rc = filter(c))) return rc;
                if ((rc = kscf_rr(s, c))) return rc;
            }
    }
    return kscf_post(s, res);
}

int hub_kscf_iterate_batch(int nobj, hub_kscf_t* objs, hub_scf_result* res, void* cuda_stream) {
    hub::NvtxRange nvtx_("hub_kscf_iterate_batch");
    if (nobj < 1 || !objs || !res) return HUB_EINVAL;
    for (int i = 0; i < nobj; ++i) {
        if (!objs[i]) return HUB_EINVAL;
        for (int j = 0; j < i; ++j)
            if (objs[j] == objs[i]) return HUB_EINVAL;
    }
    int rc;
    std::vector<int> active;
    for (int i = 0; i < nobj; ++i)
        if (!objs[i]->last.converged || objs[i]->iter == 0) active.push_back(i);
    for (int i : active)
        if ((rc = kscf_set_D(objs[i]))) return rc;
    int maxpass = 0;
    for (int i : active) maxpass = std::max(maxpass, kscf_passes(objs[i]));
    for (int pass = 0; pass < maxpass; ++pass)
        for (int sp = 0; sp < 2; ++sp) {
            // every channel of this spin still due a pass, one graph for all of them
            std::vector<std::pair<int, int>> ch;       // (object, channel)
            for (int i : active) {
                hub_kscf_t s = objs[i];
                if (sp >= s->p.nspin || pass >= kscf_passes(s)) continue;
                for (int k = 0; k < s->nk; ++k) ch.emplace_back(i, sp * s->nk + k);
            }
            if (ch.empty()) continue;
            std::vector<hub_t> hs;
            std::vector<int> spin, ncol, ld;
            std::vector<void*> X;
            std::vector<double> a, b, al;
            for (auto& q : ch) {
                hub_kscf_t s = objs[q.first];
                if ((rc = kscf_bounds(s, q.second))) return rc;
                hs.push_back(s->hubs[q.second % s->nk]);
                spin.push_back(sp);
                X.push_back(s->X[q.second]);
                ncol.push_back(s->p.ncol);
                ld.push_back(s->p.ld);
                al.push_back(s->bounds[q.second][0]);
                a.push_back(s->bounds[q.second][1]);
                b.push_back(s->bounds[q.second][2]);
            }
            const int degree = objs[ch[0].first]->p.degree;
            for (auto& q : ch)
                if (objs[q.first]->p.degree != degree)
                    return kfail(objs[q.first], HUB_EINVAL, "batched SCFs need one Chebyshev degree");
            if ((rc = hub_batch_filter((int)ch.size(), hs.data(), spin.data(), X.data(), ncol.data(), ld.data(), degree,
                                       a.data(), b.data(), al.data(), cuda_stream))) {
                const char* m = hub_last_error(hs[0]);
                return kfail(objs[ch[0].first], rc, std::string("hub_batch_filter: ") + (m ? m : ""));
            }
            // spin 0 of a two-spin object waits for its spin 1 filter: both Rayleigh-Ritz
            // projections in one eigensolver launch
            for (auto& q : ch) {
                hub_kscf_t s = objs[q.first];
                if (s->p.nspin == 2 && sp == 0) continue;
                if (s->p.nspin == 2) {
                    if ((rc = kscf_rr_pair(s, q.second - s->nk))) return rc;
                } else if ((rc = kscf_rr(s, q.second))) {
                    return rc;
                }
            }
        }
    for (int i = 0; i < nobj; ++i) {
        if (std::find(active.begin(), active.end(), i) == active.end()) { res[i] = objs[i]->last; continue; }
        if ((rc = kscf_post(objs[i], &res[i]))) return rc;
    }
    return HUB_OK;
}

int hub_kscf_run_batch(int nobj, hub_kscf_t* objs, hub_scf_result* res, void* cuda_stream) {
    if (nobj < 1 || !objs || !res) return HUB_EINVAL;
    int max_iter = 0;
    for (int i = 0; i < nobj; ++i) {
        if (!objs[i]) return HUB_EINVAL;
        max_iter = std::max(max_iter, objs[i]->p.max_iter);
    }
    for (int it = 0; it < max_iter; ++it) {
        bool done = true;
        for (int i = 0; i < nobj; ++i)
            if (!(objs[i]->iter > 0 && objs[i]->last.converged) && objs[i]->iter < objs[i]->p.max_iter) done = false;
        if (done) break;
        const int rc = hub_kscf_iterate_batch(nobj, objs, res, cuda_stream);
        if (rc) return rc;
    }
    for (int i = 0; i < nobj; ++i)
        if (!res[i].converged) return kfail(objs[i], HUB_ENOCONV, "k-point SCF reached max_iter");
    return HUB_OK;
}

int hub_kscf_run(hub_kscf_t s, hub_scf_result* res) {
    if (!s) return HUB_EINVAL;
    hub_scf_result r{};
    while (s->iter < s->p.max_iter) {
        const int rc = hub_kscf_iterate(s, &r);
        if (rc) return rc;
        if (r.converged) break;
    }
    if (res) *res = r;
    return r.converged ? HUB_OK : kfail(s, HUB_ENOCONV, "k-point SCF reached max_iter");
}

int hub_kscf_get(hub_kscf_t s, double* eig, double* occ, double* D_re, double* D_im) {
    if (!s) return HUB_EINVAL;
    if (eig) std::copy(s->eig.begin(), s->eig.end(), eig);
    if (occ) std::copy(s->occ.begin(), s->occ.end(), occ);
    if (D_re) std::copy(s->Dr_out.begin(), s->Dr_out.end(), D_re);
    if (D_im) std::copy(s->Di_out.begin(), s->Di_out.end(), D_im);
    return HUB_OK;
}

}  // extern "C"
