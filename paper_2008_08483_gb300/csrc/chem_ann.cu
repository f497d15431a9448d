// chem_ann.cu -- C ABI of the approximate-ANN equilibrium constants (Sec. 2.3, Eqs. 12-14)
// and of the exact ln K_c table that trains them (Eqs. 8-11).
#include <math.h>
#include <string.h>

#include <vector>

#include "chem_internal.h"

struct chem_kc_ann {
    const chem_mech *mech;
    int device;
    void *d_blob;
    chem::KcAnnView view;
};

using namespace chem;

static chem_status check_dev(const chem_mech *m)
{
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != m->device) return set_error(CHEM_EINVAL, "mechanism lives on device %d", m->device);
    return CHEM_OK;
}

extern "C" chem_status chem_log_kc(const chem_mech *m, int64_t n, const double *T, double *lnkc,
                                   int64_t ldK, void *stream)
{
    clear_error();
    if (!m) return set_error(CHEM_EINVAL, "mechanism is NULL");
    if (n < 0) return set_error(CHEM_EINVAL, "n < 0");
    if (ldK < m->nr) return set_error(CHEM_EINVAL, "ldK below n_reactions=%d", m->nr);
    if (n == 0) return CHEM_OK;
    if (!T || !lnkc) return set_error(CHEM_EINVAL, "NULL T or lnKc");
    chem_status st = check_dev(m);
    if (st != CHEM_OK) return st;
    return launch_log_kc(m, n, T, lnkc, ldK, (cudaStream_t)stream);
}

extern "C" chem_status chem_kc_ann_load(const chem_mech *m, const chem_kc_ann_desc *d,
                                        chem_kc_ann **out)
{
    clear_error();
    if (!out) return set_error(CHEM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!m || !d) return set_error(CHEM_EINVAL, "NULL mechanism or descriptor");
    const int nl = d->n_layers, nh = d->n_hidden, nr = m->nr;
    if (nl < 1 || nl > 8) return set_error(CHEM_EINVAL, "n_layers must be 1..8");
    if (nh < 1 || nh > kAnnMaxHidden) return set_error(CHEM_EINVAL, "n_hidden must be 1..%d", kAnnMaxHidden);
    if (d->activation != CHEM_ACT_RELU && d->activation != CHEM_ACT_ELU)
        return set_error(CHEM_EINVAL, "unknown activation %d", d->activation);
    if (!(d->x_std > 0.0f) || !isfinite(d->x_mean))
        return set_error(CHEM_EINVAL, "x_std must be > 0 and x_mean finite");
    if (!d->w_in || !d->b_in || !d->w_out || !d->b_out || !d->y_mean || !d->y_std ||
        (nl > 1 && (!d->w_hid || !d->b_hid)))
        return set_error(CHEM_EINVAL, "NULL weight array");
    chem_status st = check_dev(m);
    if (st != CHEM_OK) return st;
    // one blob: w_in, b_in, w_hid, b_hid, w_out, b_out, y_mean, y_std
    const size_t n_in = nh, n_hid = (size_t)(nl - 1) * nh * nh, n_bh = (size_t)(nl - 1) * nh;
    const size_t n_out = (size_t)nr * nh;
    std::vector<float> h;
    h.reserve(2 * n_in + n_hid + n_bh + n_out + 3 * (size_t)nr);
    auto put = [&](const float *p, size_t cnt) {
        for (size_t i = 0; i < cnt; ++i) h.push_back(p ? p[i] : 0.0f);
    };
    put(d->w_in, n_in);
    put(d->b_in, n_in);
    // hidden weights stored input-major per layer ([n_layers - 1][input][output]): lane o of
    // the FP32 kernel computes output unit o, so one input's weights are read together
    for (int l = 0; l + 1 < nl; ++l)
        for (int i = 0; i < nh; ++i)
            for (int o = 0; o < nh; ++o)
                h.push_back(d->w_hid[((size_t)l * nh + o) * nh + i]);
    put(d->b_hid, n_bh);
    // output weights stored hidden-unit-major ([n_hidden][n_reactions]): the FP32 kernel's
    // lanes take consecutive reactions and read one hidden unit's weights together
    for (int u = 0; u < nh; ++u)
        for (int j = 0; j < nr; ++j) h.push_back(d->w_out[(size_t)j * nh + u]);
    put(d->b_out, nr);
    put(d->y_mean, nr);
    put(d->y_std, nr);
    for (float v : h)
        if (!isfinite(v)) return set_error(CHEM_EINVAL, "non-finite weight");
    chem_kc_ann *a = new (std::nothrow) chem_kc_ann();
    if (!a) return set_error(CHEM_ENOMEM, "host allocation failed");
    a->mech = m;
    a->device = m->device;
    cudaError_t e = cudaMalloc(&a->d_blob, h.size() * sizeof(float));
    if (e != cudaSuccess) {
        delete a;
        return set_error(CHEM_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(a->d_blob, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(a->d_blob);
        delete a;
        return set_error(CHEM_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    const float *b = (const float *)a->d_blob;
    KcAnnView &v = a->view;
    v.nl = nl;
    v.nh = nh;
    v.act = d->activation;
    v.x_mean = d->x_mean;
    v.x_inv_std = 1.0f / d->x_std;
    v.w_in = b;
    v.b_in = b + n_in;
    v.w_hid = b + 2 * n_in;
    v.b_hid = v.w_hid + n_hid;
    v.w_out = v.b_hid + n_bh;
    v.b_out = v.w_out + n_out;
    v.y_mean = v.b_out + nr;
    v.y_std = v.y_mean + nr;
    *out = a;
    return CHEM_OK;
}

extern "C" chem_status chem_kc_ann_free(chem_kc_ann *a)
{
    clear_error();
    if (!a) return CHEM_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != a->device) cudaSetDevice(a->device);
    cudaDeviceSynchronize();
    cudaError_t e = cudaFree(a->d_blob);
    if (cur >= 0 && cur != a->device) cudaSetDevice(cur);
    delete a;
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "cudaFree: %s", cudaGetErrorString(e));
    return CHEM_OK;
}

extern "C" chem_status chem_source_term_kc_ann(const chem_mech *m, const chem_kc_ann *a, int64_t n,
                                               const float *T, const float *P, const float *Y,
                                               int64_t ldY, float *omega, int64_t ldO,
                                               void *stream)
{
    clear_error();
    if (!m) return set_error(CHEM_EINVAL, "NULL mechanism");
    if (a && a->mech != m) return set_error(CHEM_EINVAL, "the network was built for another mechanism");
    if (n < 0) return set_error(CHEM_EINVAL, "n_cells < 0");
    if (ldY < m->ns || ldO < m->ns) return set_error(CHEM_EINVAL, "ldY / ldO below n_species");
    if (n == 0) return CHEM_OK;
    if (!T || !P || !Y || !omega) return set_error(CHEM_EINVAL, "NULL array with n_cells > 0");
    chem_status st = check_dev(m);
    if (st != CHEM_OK) return st;
    if (!a) return launch_source_fp32_warp(m, n, T, P, Y, ldY, omega, ldO, (cudaStream_t)stream);
    return launch_source_fp32_ann(m, a->view, n, T, P, Y, ldY, omega, ldO, (cudaStream_t)stream);
}
