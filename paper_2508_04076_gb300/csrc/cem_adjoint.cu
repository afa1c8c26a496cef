// Discrete adjoint of the explicit step (fixed topology): gradients of
//   J = c * 1/2 u_N^T K u_N + w . u_N
// with respect to every input element's Young's modulus and the traction
// amplitude alpha (f_ext = alpha f_ext, at alpha = 1).
//
// The step x_n = (u, v, a) -> x_{n+1} of Eqs. 13-15 with a' = M^-1 (f - K u')
// has the reverse sweep
//   g = la + dt/2 lv,  y = M^-1 g,  lu' = lu - K y,
//   (lu, lv, la) <- (lu', lv + dt lu', dt/2 lv + dt^2/2 lu'),
//   dJ/dE_j -= y^T (dK/dE_j) u_{n+1} = (V_j/6) sum_{k in edges(j)} epsbar_k(y)^T Dhat epsbar_k(u_{n+1}),
//   dJ/dalpha += y . f_ext,
// started from lu = c K u_N + w, lv = la = 0; a run from step 0 adds the
// dependence of a_0 = alpha M^-1 f_ext.  K is symmetric, so K y is the
// ordinary internal-force evaluation applied to y.
//
// Memory: states (u, v, a) are kept every C steps (C = ceil(sqrt(n)) unless
// given); each segment is re-run forward, storing its displacements, before
// its reverse sweep, so the working set is O((n / C + C) N) instead of O(n N).
#include "cem_common.cuh"

#include <cmath>
#include <vector>

namespace {

struct Pool {
    cem_ctx* c;
    std::vector<void*> ptrs;
    template <class T>
    T* get(int64_t n) {
        size_t bytes = ((size_t)std::max<int64_t>(n, 1) * sizeof(T) + 255) & ~(size_t)255;
        void* p = nullptr;
        if (c->alloc) p = c->alloc(bytes, (void*)c->stream, c->alloc_user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (p) ptrs.push_back(p);
        return (T*)p;
    }
    ~Pool() {
        cudaStreamSynchronize(c->stream);
        for (void* p : ptrs) {
            if (c->free_fn) c->free_fn(p, (void*)c->stream, c->alloc_user);
            else cudaFree(p);
        }
    }
};

int copy3(cem_ctx* c, double* dst, const double* src) {   // [3][Nc] vector, first N entries of each row
    for (int k = 0; k < 3; ++k)
        CEM_CK(c, cudaMemcpyAsync(dst + k * c->Nc, src + k * c->Nc, c->N * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->stream));
    return CEM_OK;
}

}  // namespace

extern "C" int cem_adjoint(cem_ctx* c, int64_t n_steps, int64_t checkpoint_every, double c_strain,
                           const double* w_u, double* J, double* dJ_dE, double* dJ_dalpha) {
    if (!c || n_steps < 0 || !J || !dJ_dE || !dJ_dalpha) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called first");
    if (c->split_enabled) return cem_fail(c, CEM_ESTATE, "the adjoint needs a fixed topology (split_enabled = 0)");
    if (c->n_inst > 1) return cem_fail(c, CEM_ESTATE, "the adjoint takes one specimen, not an ensemble");
    if (c->n_dir > 0) return cem_fail(c, CEM_ESTATE, "the adjoint does not take prescribed velocities");
    if (c->elem_type != CEM_ELEM_TET4) return cem_fail(c, CEM_ESTATE, "the adjoint covers tetrahedral meshes");
    CEM_CK(c, cudaSetDevice(c->device));
    const int64_t C = checkpoint_every > 0 ? checkpoint_every
                                           : std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)n_steps)));
    const int64_t n_ck = n_steps > 0 ? (n_steps + C - 1) / C : 0;
    const bool from_start = c->step == 0;
    const int64_t Nc = c->Nc, N = c->N, Tc = c->Tc;
    Pool pool{c, {}};
    double* lu = pool.get<double>(3 * Nc);
    double* lv = pool.get<double>(3 * Nc);
    double* la = pool.get<double>(3 * Nc);
    double* y = pool.get<double>(3 * Nc);
    double* Ky = pool.get<double>(3 * Nc);
    double* w = pool.get<double>(3 * Nc);
    double* s = pool.get<double>(c->Ec);
    double* gE = pool.get<double>(Tc);
    double* dal = pool.get<double>(n_steps + 2);
    double* ck = pool.get<double>(std::max<int64_t>(n_ck, 1) * 9 * Nc);
    double* fin = pool.get<double>(9 * Nc);
    double* seg = pool.get<double>(std::max<int64_t>(std::min(C, n_steps), 1) * 3 * Nc);
    const bool mixed = c->precision == CEM_MIXED;
    void* h2 = mixed ? (void*)pool.get<float>(8 * Tc) : (void*)pool.get<double>(6 * Tc);
    float* yhl = mixed ? pool.get<float>(8 * Nc) : nullptr;
    if (!lu || !lv || !la || !y || !Ky || !w || !s || !gE || !dal || !ck || !fin || !seg || !h2 || (mixed && !yhl))
        return cem_fail(c, CEM_ENOMEM, "adjoint working memory");
    cudaStream_t st = c->stream;
    CEM_CK(c, cudaMemsetAsync(gE, 0, Tc * sizeof(double), st));
    CEM_CK(c, cudaMemsetAsync(w, 0, 3 * Nc * sizeof(double), st));
    CEM_CK(c, cudaMemsetAsync(dal, 0, (n_steps + 2) * sizeof(double), st));
    if (w_u) {   // host N x 3 row-major -> device [3][Nc]
        std::vector<double> t(3 * N);
        for (int64_t i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) t[k * N + i] = w_u[3 * i + k];
        for (int k = 0; k < 3; ++k)
            CEM_CK(c, cudaMemcpyAsync(w + k * Nc, t.data() + k * N, N * sizeof(double), cudaMemcpyHostToDevice, st));
        CEM_CK(c, cudaStreamSynchronize(st));
    }
    const int64_t step0 = c->step;
    int rc;
    auto save = [&](double* dst) {
        int r;
        if ((r = copy3(c, dst, c->u)) || (r = copy3(c, dst + 3 * Nc, c->v)) || (r = copy3(c, dst + 6 * Nc, c->a)))
            return r;
        return (int)CEM_OK;
    };
    auto restore = [&](const double* src) {
        int r;
        if ((r = copy3(c, c->u, src)) || (r = copy3(c, c->v, src + 3 * Nc)) || (r = copy3(c, c->a, src + 6 * Nc)))
            return r;
        return cem_launch_pred_u(c);
    };
    // forward sweep with checkpoints
    for (int64_t n = 0; n < n_steps; ++n) {
        if (n % C == 0 && (rc = save(ck + (n / C) * 9 * Nc))) return rc;
        if ((rc = cem_run_step(c))) return rc;
    }
    if ((rc = save(fin))) return rc;
    // terminal: J, lu = c K u_N + w, explicit dJ/dE of the strain-energy term
    if ((rc = cem_adj_apply_K(c, c->u, yhl, Ky))) return rc;
    if ((rc = cem_adj_dot(c, c->u, Ky, nullptr, dal + n_steps)) || (rc = cem_adj_dot(c, w, c->u, nullptr, dal + n_steps + 1)))
        return rc;
    if ((rc = cem_adj_init(c, lu, lv, la, Ky, w, c_strain))) return rc;
    if ((rc = cem_adj_strain(c, c->u, yhl, h2))) return rc;
    if ((rc = cem_adj_grad_E(c, h2, h2, s, 0.5 * c_strain, gE))) return rc;
    std::vector<double> jparts(2);
    CEM_CK(c, cudaMemcpyAsync(jparts.data(), dal + n_steps, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CEM_CK(c, cudaStreamSynchronize(st));
    // reverse sweep, one checkpoint segment at a time
    for (int64_t k = n_ck - 1; k >= 0; --k) {
        const int64_t s0 = k * C, s1 = std::min(n_steps, s0 + C);
        if ((rc = restore(ck + k * 9 * Nc))) return rc;
        c->step = step0 + s0;
        for (int64_t n = s0; n < s1; ++n) {
            if ((rc = cem_run_step(c))) return rc;
            if ((rc = copy3(c, seg + (n - s0) * 3 * Nc, c->u))) return rc;
        }
        for (int64_t n = s1 - 1; n >= s0; --n) {
            const double* un1 = seg + (n - s0) * 3 * Nc;   // u_{n+1}
            if ((rc = cem_adj_y(c, la, lv, y, dal + n))) return rc;
            if ((rc = cem_adj_strain(c, un1, mixed ? c->uhl : nullptr, h2))) return rc;
            if ((rc = cem_adj_apply_K(c, y, yhl, Ky))) return rc;
            if ((rc = cem_adj_grad_E(c, mixed ? (void*)c->h32 : (void*)c->h, h2, s, -1.0, gE))) return rc;
            if ((rc = cem_adj_update(c, lu, lv, la, Ky))) return rc;
        }
    }
    double a0term = 0.0;
    if (from_start) {
        if ((rc = cem_adj_dot(c, la, c->fext, c->minv, dal + n_steps))) return rc;
        CEM_CK(c, cudaMemcpyAsync(&a0term, dal + n_steps, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    // leave the context at the end of the forward run
    if ((rc = restore(fin))) return rc;
    c->step = step0 + n_steps;
    // outputs
    std::vector<double> dsteps(std::max<int64_t>(n_steps, 1)), g(c->T);
    std::vector<int> anc(c->T);
    std::vector<uint8_t> act(c->T);
    if (n_steps > 0)
        CEM_CK(c, cudaMemcpyAsync(dsteps.data(), dal, n_steps * sizeof(double), cudaMemcpyDeviceToHost, st));
    CEM_CK(c, cudaMemcpyAsync(g.data(), gE, c->T * sizeof(double), cudaMemcpyDeviceToHost, st));
    CEM_CK(c, cudaMemcpyAsync(anc.data(), c->anc, c->T * sizeof(int), cudaMemcpyDeviceToHost, st));
    CEM_CK(c, cudaMemcpyAsync(act.data(), c->active, c->T, cudaMemcpyDeviceToHost, st));
    CEM_CK(c, cudaStreamSynchronize(st));
    *J = c_strain * 0.5 * jparts[0] + jparts[1];
    double da = 0.0;
    for (int64_t n = 0; n < n_steps; ++n) da += dsteps[n];
    *dJ_dalpha = da + a0term;
    for (int64_t t = 0; t < c->T0; ++t) dJ_dE[t] = 0.0;
    for (int64_t j = 0; j < c->T; ++j)   // a sub-element carries its parent's modulus
        if (act[j]) dJ_dE[anc[j]] += g[j];
    return CEM_OK;
}
