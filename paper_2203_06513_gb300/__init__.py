"""GB300-native energy-conserving PIC (1D reduced relativistic Vlasov--Maxwell).

The compute path is the C-ABI library ``libpic`` (CUDA, sm_103a) declared in
``include/pic.h``; ``paper_2203_06513_gb300.pic`` is its thin ctypes binding and
``paper_2203_06513_gb300.inputs`` the seeded workload generator.  Importing the
package does not load the CUDA library; ``pic.load()`` does, and fails loudly
when it is missing.
"""
__all__ = ["inputs", "pic"]
