// Host-side state of a realisation (pe_ctx), shared by the context and batch code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pepic.h"

#define PE_TRY(x)                     \
    do {                              \
        int _rc = (x);                \
        if (_rc != PE_OK) return _rc; \
    } while (0)

struct pe_ctx {
    pe_config cfg;
    pe_layout lay;
    char* arena;
    cudaStream_t stream;
    double dx;
    int s_w, s_p, nc;
    int bin_shift;       // Haar: restriction samples summed over coarse bins; else 0
    int nb;              // sample length per moment: ncell >> bin_shift
    int ps;              // phase-space coarse variable (PE_COARSE_PHASE_SPACE)
    int pres;            // ion pressure active (PE_COARSE_MOMENTS_PRESSURE): three nodal moments
    int s_e;             // second-moment fixed-point shift (pres)
    int K_cur;           // burst length of the next bursts (the configured K unless adapted)
    int te_active;       // kinetic electrons: their kinetic energy is an active variable
    double* we;          // te_active: [K+2] sampled energies, then the projected energy and its slope
    double te;           // T_e / T_e0 of the last lift
    double we_ref;       // the electrons' kinetic energy at the initial load (T_e = T_e0)
    double we_last;      // the projected energy read at the last lift
    int nv;              // velocity cells (phase space; the fine cells n_vf of the wavelet form)
    int psw;             // phase space, wavelet form: hat rows in x, DWT in v to nvc coefficients
    int nvc;             // wavelet form: velocity coefficients per coarse node
    double* ps_hist;     // wavelet form: [n_coarse][nv] lifted histograms
    float* ps_node_table;  // wavelet form: [ncell][3 nv + 1] fine-node sampling rows
    float* ps_node_dens;   // wavelet form: [ncell] fine-node densities
    double vmin, dv;     // velocity cells: [vmin + j dv, vmin + (j+1) dv)
    int64_t ncoef;       // active coarse coefficients: 2 n_coarse or n_coarse n_v
    int64_t row_fx;      // int64 words per restriction-sample row
    int64_t crow;        // doubles per coarse-sample row
    double* ps_mass;     // [n_coarse]
    double* ps_cdf;      // [n_coarse][n_v + 1]
    double* ps_scratch;  // [2 n_coarse (n_v + 1)]
    float* ps_table;     // [n_coarse][3 n_v + 1] FP32 sampling rows
    int32_t* ps_flags;
    int walls;           // bounded grid (PE_BOUNDARY_ABSORBING)
    int phi_hist;        // phi and phi + ncell hold two solutions one fine step apart
    void* eq_scratch;    // equal-weight loading scratch (bounded grids)
    int bank;            // which particle bank is current
    int v_at_integer;    // stored v is at integer time
    int fresh;           // particles were just loaded/lifted (not yet advanced)
    int rho_valid;       // rho holds the deposit of the current particles
    int64_t macro_steps, fine_steps;
    double time;
    double dT_cur;       // Delta t of the next macro step (the configured one unless set or adapted)
    int coarse_state;    // the coarse state (not the particles) is the state: after a projection,
                         // pe_set_coarse or a restore; 0 after a load or plain PIC
    int32_t* cell[2];
    float* theta[2];
    float* v[2];
    float* w[2];
    int64_t* rho;
    // kinetic electrons (PE_ELECTRONS_KINETIC)
    int kinetic;
    double qm_e, v_th_e;
    int ebank;           // which electron bank is current
    int e_v_at_integer;  // stored electron v is at integer time
    int32_t* ecell[2];
    float* etheta[2];
    float* ev[2];
    float* ew[2];
    int64_t* rho_e;
    double* phi;
    double* E;
    float* Ef;
    float* E0f;
    int64_t* samples;  // [K+2][2][ncell]; row K+1 is measurement scratch
    double* csamples;  // [K+2][2][nc]
    double* coarse;
    double* slope;
    float* prof;
    int32_t* sort;
    uint32_t* status;
    int32_t* diag;
    // kernel timing (pe_profile): start/stop event pairs per launch kind (PE_PROF_*)
    int profiling;
    std::vector<cudaEvent_t>* prof_ev[PE_PROF_NKINDS];
    size_t prof_n[PE_PROF_NKINDS];  // pairs recorded since the last read
};


// Internal helpers of the context API used by the batch code (pe_capi.cu).
int pe_ctx_field_solve(pe_ctx* x);
uint64_t pe_ctx_lift_seed(const pe_ctx* x);
int pe_ctx_burst_range(pe_ctx* x, int p_begin, int p_end, int final_sample);
