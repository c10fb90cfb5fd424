"""GB300-native listmode SPDHG (LM-SPDHG) for sparse Poisson TOF PET data.

Submodules:
  synth  - seeded synthetic inputs (scanner, phantom, Monte Carlo events)
  lm     - binding of the C-ABI library liblmspdhg.so (CUDA, sm_103a)

A reconstruction through the binding (every step runs in the library's
kernels; torch tensors only hold device memory):

    from paper_2201_05497_gb300 import build, lm, synth
    build.build(); lm.load_library()
    wl = synth.workload("3d_short")
    geo = lm.Geometry.from_workload(wl)
    sens = lm.sens(geo, lor_factor)                       # P^T 1
    pe = lm.event_setup(geo, lm.DeviceEvents(...), n)     # mu, every n-th event to sub list n
    x0 = ...                                              # e.g. lm.emtv_epoch(...) (Alg. 3 warm start)
    st = lm.LMSPDHG(geo, pe, sens, x0, beta=0.03, n_subsets=n, knorm=lm.knorm_fp64(geo, 1000))
    for seq in sequences:                                 # 2n selections per epoch
        st.epoch(seq)
    x = st.x()

Options of LMSPDHG: the directional TV prior (xi=lm.dtv_field(geo, v, eta)),
the image-space resolution model (res_fwhm, with sens = lm.res_apply(geo, fwhm,
sens)), sinogram SPDHG (sinogram=1 with lm.sino_setup, 2 with lm.sino_count),
the deterministic back-projection, and lm.Batch / lm.Server for many frames.
"""
