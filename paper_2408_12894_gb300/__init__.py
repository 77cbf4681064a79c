"""GB300-native FLoD splatting path: a C-ABI CUDA library (sm_103a) and its Python binding.

* ``synth``   -- seeded synthetic scenes, cameras and job mixes (inputs only).
* ``flod``    -- ctypes binding of the C-ABI (``flod_preprocess``, ``flod_bin_sort``,
                 ``flod_render_fwd``, ``flod_render_bwd``, ``flod_select_levels``,
                 ``flod_adjust_scale``) plus a torch.autograd.Function over it.
* ``_build``  -- compiles the library for sm_103a in-tree.

The binding loads the compiled library on first use and raises if it is missing: there is
no CPU fallback.
"""
