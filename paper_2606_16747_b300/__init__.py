"""STAR-NT neural order-independent transparency: B300-native per-frame hot path."""
