"""FP64 CPU oracle of the Dynamic DH-MBIR step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this
package; the GPU library never does.
"""
