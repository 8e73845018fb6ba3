"""Seeded synthetic inputs (detector, events, raw banks) shared by every consumer."""
from .generator import (Batch, Geometry, CONFIGS, generate, generate_config, encode, subset,
                        AlignmentSet, generate_alignment,
                        Z_LAYERS, STEREO_DEG, SECTOR_PITCH, STRIP_PITCH, N_STRIPS, Z_VELO,
                        Z_KINK, KICK_K, tan_stereo_f32, KickMap, field_kick, kick_map)
from .params import CompassParams
